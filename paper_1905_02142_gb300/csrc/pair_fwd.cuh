// Forward pair kernel: expansion coefficients c_nlm of every atom (Sec. II, Eqs. 01/08,
// summed over neighbours, plus the central atom).
//
// One warp per atom.  The atom's neighbours of one species are taken 32 at a time, one
// per lane: the lane evaluates its neighbour's radial coefficients b_n (table path:
// cubic-Hermite interpolation of FP64-built nodes; recursion path: Eq. 04 per pair in
// FP64) and the angular factors a_lm = 4 pi ilexp_l(z) Y_lm(r_hat) (real Y_lm from a
// pole-free recurrence), and stages them in shared memory.  The warp then contracts the
// batch, c[n][lm] += sum_k b_n(k) a_lm(k), with every lane owning the columns
// lm = lane + 32 j for all n, so the sum over neighbours is a register accumulation
// with no atomics.  The recursion path accumulates in the primitive basis and applies
// W = S^-1/2 per atom at the end (Sec. III.A: work in the alpha basis, then transform).
#pragma once
#include "internal.h"
#include "soapmath.cuh"
#include "table.cuh"

template <typename T> __device__ __forceinline__ T sq(T x) { return x * x; }

template <typename T, int NC, int LC, bool TABLE>
__global__ void __launch_bounds__(SG_WARPS * 32)
pair_fwd_kernel(const FwdArgs<T> a) {
  constexpr int LCC = (LC + 1) * (LC + 1);
  constexpr int LPL = (LCC + 31) / 32;
  constexpr int AS = (LCC % 2 == 0) ? LCC + 1 : LCC;
  constexpr int NP = (NC + 3) / 4 * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* a_s = reinterpret_cast<T*>(smem_raw) + warp * (32 * AS + 32 * NP);
  T* b_s = a_s + 32 * AS;
  const int L = (a.lmax + 1) * (a.lmax + 1);
  const int nch = a.nsp * a.nmax;
  const T FOUR_PI = (T)12.566370614359172;

  for (int atom = blockIdx.x * SG_WARPS + warp; atom < a.n_atoms; atom += gridDim.x * SG_WARPS) {
    const int spc = a.species[atom];
    for (int s = 0; s < a.nsp; ++s) {
      const int beg = a.seg_offs[atom * a.nsp + s];
      const int end = a.seg_offs[atom * a.nsp + s + 1];
      T acc[NC][LPL];
#pragma unroll
      for (int n = 0; n < NC; ++n)
#pragma unroll
        for (int j = 0; j < LPL; ++j) acc[n][j] = T(0);

      for (int base = beg; base < end; base += 32) {
        const int pidx = base + lane;
        if (pidx < end) {
          const Vec4<T> v = a.pair_r[a.pair_idx ? a.pair_idx[pidx] : pidx];
          // |r| < 0 marks a pair beyond r_cut in a list built with a skin: no contribution
          const bool live = v.w >= T(0);
          const T r = live ? v.w : T(1), inv = T(1) / r;
          const T ux = live ? v.x * inv : T(0), uy = live ? v.y * inv : T(0), uz = live ? v.z * inv : T(1);
          T bn[NC], il[LC + 1];
          if constexpr (TABLE) {
            float f[NC + LC + 1];
            table_interp<NC, LC, false>(a.table, a.ti, (float)r, f, nullptr);
#pragma unroll
            for (int n = 0; n < NC; ++n) bn[n] = f[n];
#pragma unroll
            for (int l = 0; l <= LC; ++l) il[l] = f[NC + l];
          } else {
            double ba[NC];
            radial_alpha<double, NC>((double)r, a.p, ba);
            double spp = a.p.s0p + a.p.ap * (double)r;
            double ild[LC + 1];
            ilexp_all<double, LC>((double)r * (double)r / (spp * spp), ild);
#pragma unroll
            for (int n = 0; n < NC; ++n) bn[n] = (T)ba[n];
#pragma unroll
            for (int l = 0; l <= LC; ++l)
              il[l] = (l <= a.lmax) ? (T)(ild[l] * (a.p.eq08 ? (2.0 * l + 1.0) : 1.0)) * FOUR_PI : T(0);
          }
#pragma unroll
          for (int n = 0; n < NP; ++n) b_s[lane * NP + n] = (n < NC && live) ? bn[n] : T(0);
          T* arow = a_s + lane * AS;
          for_each_ylm<T, LC>(ux, uy, uz, a.yc, [&](int l, int m, T y) { arow[lm_index(l, m)] = il[l] * y; });
        }
        __syncwarp();
        const int cnt = min(32, end - base);
        for (int k = 0; k < cnt; ++k) {
          T bk[NP];
          if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int n = 0; n < NP; n += 4) {
              float4 t4 = *reinterpret_cast<const float4*>(b_s + k * NP + n);
              bk[n] = t4.x; bk[n + 1] = t4.y; bk[n + 2] = t4.z; bk[n + 3] = t4.w;
            }
          } else {
#pragma unroll
            for (int n = 0; n < NP; n += 2) {
              double2 t2 = *reinterpret_cast<const double2*>(b_s + k * NP + n);
              bk[n] = t2.x; bk[n + 1] = t2.y;
            }
          }
          const T* arow = a_s + k * AS;
#pragma unroll
          for (int j = 0; j < LPL; ++j) {
            const int lm = lane + 32 * j;
            const T av = (lm < LCC) ? arow[lm] : T(0);
#pragma unroll
            for (int n = 0; n < NC; ++n) acc[n][j] = fma(bk[n], av, acc[n][j]);
          }
        }
        __syncwarp();
      }
      if (s == spc && lane == 0) {
#pragma unroll
        for (int n = 0; n < NC; ++n) acc[n][0] += a.bc.cen[n];
      }
#pragma unroll
      for (int n = 0; n < NC; ++n) {
        if (n < a.nmax) {
          T out[LPL];
#pragma unroll
          for (int j = 0; j < LPL; ++j) {
            if constexpr (TABLE) {
              out[j] = acc[n][j];
            } else {
              T o = T(0);
#pragma unroll
              for (int al = 0; al < NC; ++al) o = fma(a.bc.W[n][al], acc[al][j], o);
              out[j] = o;
            }
          }
          T* crow = a.c + ((size_t)atom * nch + s * a.nmax + n) * L;
#pragma unroll
          for (int j = 0; j < LPL; ++j) {
            const int lm = lane + 32 * j;
            if (lm < L) crow[lm] = out[j];
          }
        }
      }
    }
  }
}

template <typename T, int NC, int LC, bool TABLE>
static cudaError_t launch_fwd(const FwdArgs<T>& a, cudaStream_t st) {
  constexpr int LCC = (LC + 1) * (LC + 1);
  constexpr int AS = (LCC % 2 == 0) ? LCC + 1 : LCC;
  constexpr int NP = (NC + 3) / 4 * 4;
  const size_t smem = (size_t)SG_WARPS * (32 * AS + 32 * NP) * sizeof(T);
  auto kern = pair_fwd_kernel<T, NC, LC, TABLE>;
  cudaError_t e = sg_set_smem<pair_fwd_kernel<T, NC, LC, TABLE>>(smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SG_WARPS * 32, smem);
  if (per_sm < 1) per_sm = 1;
  long long need = (a.n_atoms + SG_WARPS - 1) / SG_WARPS;
  long long grid = (long long)sms * per_sm * 4;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, SG_WARPS * 32, smem, st>>>(a);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

template <typename T>
cudaError_t sg_pair_forward(const FwdArgs<T>& a, int cls, bool table, cudaStream_t st) {
  if (a.n_atoms == 0) return cudaSuccess;
  if (table) {
    if constexpr (sizeof(T) == 4) {
      switch (cls) {
        case 0: return launch_fwd<T, 6, 6, true>(a, st);
        case 1: return launch_fwd<T, 8, 8, true>(a, st);
        case 2: return launch_fwd<T, 10, 10, true>(a, st);
        default: return launch_fwd<T, 12, 12, true>(a, st);
      }
    }
    return cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 8) {
    switch (cls) {
      case 0: return launch_fwd<T, 6, 6, false>(a, st);
      case 1: return launch_fwd<T, 8, 8, false>(a, st);
      case 2: return launch_fwd<T, 10, 10, false>(a, st);
      default: return launch_fwd<T, 12, 12, false>(a, st);
    }
  }
  return cudaErrorInvalidValue;
}

