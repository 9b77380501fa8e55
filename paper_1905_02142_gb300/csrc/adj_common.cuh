// Helpers shared by the two tensor-core adjoint kernels of the mixed-precision path
// (pair_adj_mma.cu: mma.sync; pair_adj_tc.cu: tcgen05 with TMEM accumulators): the order in
// which the harmonic recursion visits (l, m), its packed coefficients, FP16 packing, and
// block reductions.
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

#include "internal.h"

namespace {

// Number of tau rows the recursion visits for a given l_max: the m = 0 column (l_max + 1
// entries, padded to an even count) followed by (cos, sin) pairs for m >= 1.
__host__ __device__ inline int tau_even(int lmax) { return (lmax + 2) & ~1; }
__host__ __device__ inline int tau_count(int lmax) { return tau_even(lmax) + lmax * (lmax + 1); }
__host__ __device__ inline int tau_rows16(int lmax) { return (tau_count(lmax) + 15) & ~15; }

// tau of (l, m) (m < 0: the sin-type harmonic l^2 + l + m)
__device__ __forceinline__ int tau_of(int l, int ms, int lmax) {
  if (ms == 0) return l;
  const int m = ms < 0 ? -ms : ms;
  const int base = tau_even(lmax) + 2 * ((m - 1) * (lmax + 1) - m * (m - 1) / 2);
  return base + 2 * (l - m) + (ms < 0 ? 1 : 0);
}

// Packed recursion coefficients for the rolled (l, m) loops.  For column j and degree l:
//   A(l, j) = s1[j] (l = j + 1), a[l][j] (l >= j + 2), 0 otherwise
//   B(l, j) = b[l][j] (l >= j + 2), 0 otherwise
//   C(l, j) = seed[j] (l = j), 0 otherwise
// so that N~_l^j = A z N~_{l-1}^j - B N~_{l-2}^j + C for every l >= j, starting from zeros.
template <int LC> struct CoefShared {
  float4 p[LC + 1][LC + 1];  // (A(l,m), B(l,m), A(l,m+1), B(l,m+1))
  float4 q[LC + 1][LC + 1];  // (C(l,m), C(l,m+1), d[l][m], 0)
};

__device__ __forceinline__ float coef_a(const YlmCoef<float>& y, int l, int j) {
  if (l == j + 1) return y.s1[j];
  return l >= j + 2 ? y.a[l][j] : 0.f;
}
__device__ __forceinline__ float coef_b(const YlmCoef<float>& y, int l, int j) {
  return l >= j + 2 ? y.b[l][j] : 0.f;
}
__device__ __forceinline__ float coef_c(const YlmCoef<float>& y, int l, int j) {
  return (l == j && j <= SG_MAX_LMAX) ? y.seed[j] : 0.f;
}

// 4-byte asynchronous global -> shared copy (completes at cp.async.wait_group)
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ uint32_t pack_half2(__half lo_k, __half hi_k) {
  return (uint32_t)__half_as_ushort(lo_k) | ((uint32_t)__half_as_ushort(hi_k) << 16);
}

__host__ __device__ inline int align4(int x) { return (x + 3) & ~3; }

template <int W> __device__ __forceinline__ float block_sum(float v, float* red) {
  v = warp_sum(v);
  __syncthreads();  // red free
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < W; ++w) t += red[w];
  return t;
}

template <int W> __device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < W; ++w) t = fmaxf(t, red[w]);
  return t;
}

}  // namespace
