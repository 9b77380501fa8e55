// Shared definitions of the CUDA library (device side and launch glue).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SG_MAX_NMAX 12
#define SG_MAX_LMAX 12
#define SG_MAX_SPECIES 8
#define SG_WARPS 4  // warps per block of the warp-per-atom kernels

// device-side error codes (bit flags written to the handle's error word)
#define SG_ERR_OUTSIDE_CELL 1
#define SG_ERR_COINCIDENT 2
#define SG_ERR_PAIR_CAPACITY 4
#define SG_ERR_NO_REVERSE 8
#define SG_ERR_BIN_CAPACITY 16
#define SG_ERR_TIMEOUT 32

// Hyperparameters in device form (Eq. 15, Sec. III.A-B).
struct DevParams {
  double rc, rs, s0r, s0p, ar, ap, amp_a, nf, cw;
  int nmax, lmax, nsp, eq08;
};

// A pair separation vector and its length, FP32 or FP64.
template <typename T> struct alignas(4 * sizeof(T)) Vec4 { T x, y, z, w; };

// Per-structure geometry for the neighbour builder (computed on the host in FP64).
struct StructGeom {
  double h[9];     // rows = lattice vectors
  double hinv[9];  // inverse (fractional = x @ hinv)
  float h32[9];
  float h32lo[9];  // h - (double)h32, so that h = h32 + h32lo to ~2^-48
  int nb[3];       // bins along each lattice direction
  int m[3];        // bin offsets searched: -m..m
  int bin_off;     // first bin of this structure in the flattened bin arrays
  int atom_off, n_atoms;
  float margin;    // |d2_fp32 - rc^2| below which the FP64 test decides
};

// Normalised real spherical-harmonic recurrence coefficients (fully unrolled loops index
// them with compile-time constants, so they live in the kernel parameter bank).
template <typename T> struct YlmCoef {
  T seed[SG_MAX_LMAX + 1];                 // N~_m^m (sqrt(2) folded in for m > 0)
  T s1[SG_MAX_LMAX + 1];                   // sqrt(2m+3): N~_{m+1}^m = s1[m] z N~_m^m
  T a[SG_MAX_LMAX + 1][SG_MAX_LMAX + 1];   // N~_l^m = a z N~_{l-1}^m - b N~_{l-2}^m
  T b[SG_MAX_LMAX + 1][SG_MAX_LMAX + 1];
  T d[SG_MAX_LMAX + 1][SG_MAX_LMAX + 1];   // dN~_l^m/dz = d N~_l^{m+1}
};

// W = S^-1/2 (FP64 path) and the central-atom constants.
template <typename T> struct BasisConst {
  T W[SG_MAX_NMAX][SG_MAX_NMAX];
  T cen[SG_MAX_NMAX];  // central-atom term added to c_{s_i, n, l=0, m=0}
};

__host__ __device__ inline int lm_index(int l, int m) { return l * l + l + m; }

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
