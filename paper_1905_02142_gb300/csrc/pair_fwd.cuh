// Forward pair kernel: expansion coefficients c_nlm of every atom (Sec. II, Eqs. 01/08,
// summed over neighbours, plus the central atom).
//
// One warp per atom.  The atom's neighbours of one species are taken 32 at a time, one
// per lane: the lane evaluates its neighbour's radial coefficients b_n (table path:
// cubic-Hermite interpolation of FP64-built nodes; recursion path: Eq. 04 per pair in
// FP64) and the angular factors a_lm = 4 pi ilexp_l(z) Y_lm(r_hat) (real Y_lm from a
// pole-free recurrence), and stages them in shared memory.  On the table path each lane
// first has its pair's table interval (nodes k and k + 1, 4 FP floats) bulk-copied into
// the warp's a_lm buffer, so the 32 scattered intervals of a batch arrive as 32 bulk
// copies from L2 instead of 32-way divergent loads through L1.  The warp then contracts the
// batch, c[n][lm] += sum_k b_n(k) a_lm(k), with every lane owning the columns
// lm = lane + 32 j for all n, so the sum over neighbours is a register accumulation
// with no atomics.  The recursion path accumulates in the primitive basis and applies
// W = S^-1/2 per atom at the end (Sec. III.A: work in the alpha basis, then transform).
#pragma once
#include "internal.h"
#include "soapmath.cuh"
#include "table.cuh"
#include "tcgen05.cuh"

template <typename T> __device__ __forceinline__ T sq(T x) { return x * x; }

// Shared memory of one warp, in elements of T: the a_lm rows (32 x AS), which on the table
// path first hold the 32 table intervals (32 x CS, CS = 4 FP + 4 so that the lanes' 16-byte
// reads of their own intervals fall in distinct banks), then the b_n rows (32 x NP).
template <typename T, int NC, int LC, bool TABLE> struct FwdSmem {
  static constexpr int LCC = (LC + 1) * (LC + 1);
  static constexpr int AS = (LCC % 2 == 0) ? LCC + 1 : LCC;
  static constexpr int NP = (NC + 3) / 4 * 4;
  static constexpr int CH = 4 * TableDims<NC, LC>::FP;  // floats of one interval
  static constexpr int CS = CH + 4;
  static constexpr int REG_A = (TABLE && CS > AS) ? 32 * CS : 32 * AS;
  static constexpr int WARP = REG_A + 32 * NP;
  // all warps' buffers, then one mbarrier per warp (table path)
  static constexpr size_t bytes() { return (size_t)SG_WARPS * WARP * sizeof(T) + (TABLE ? SG_WARPS * 8 : 0); }
};

template <typename T, int NC, int LC, bool TABLE>
__global__ void __launch_bounds__(SG_WARPS * 32)
pair_fwd_kernel(const FwdArgs<T> a) {
  using SM = FwdSmem<T, NC, LC, TABLE>;
  constexpr int LCC = SM::LCC;
  constexpr int LPL = (LCC + 31) / 32;
  constexpr int AS = SM::AS;
  constexpr int NP = SM::NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* a_s = reinterpret_cast<T*>(smem_raw) + warp * SM::WARP;
  T* b_s = a_s + SM::REG_A;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + (size_t)SG_WARPS * SM::WARP * sizeof(T)) + warp;
  uint32_t phase = 0;
  if constexpr (TABLE) {
    if (lane == 0) {
      tc5::mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
  }
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
        const bool has = pidx < end;
        Vec4<T> v{T(0), T(0), T(0), T(-1)};
        if (has) v = a.pair_r[a.pair_idx ? a.pair_idx[pidx] : pidx];
        // |r| < 0 marks a pair beyond r_cut in a list built with a skin: no contribution
        const bool live = v.w >= T(0);
        const T r = live ? v.w : T(1), inv = T(1) / r;
        float tt = 0.f;
        if constexpr (TABLE) {
          // this batch's table intervals into the a_lm buffer (the previous batch's reads of
          // it ended at the __syncwarp closing that batch)
          const int k = table_locate(a.ti, (float)r, tt);
          const int cnt = min(32, end - base);
          tc5::fence_proxy_async();
          if (lane == 0) tc5::mbar_expect_tx(bar, (uint32_t)(cnt * SM::CH * sizeof(float)));
          __syncwarp();
          if (has)
            tc5::bulk_load(a_s + lane * SM::CS, a.table + (size_t)k * (SM::CH / 2), SM::CH * sizeof(float), bar);
          const bool ok = __all_sync(0xffffffffu, tc5::mbar_wait(bar, phase));
          phase ^= 1;
          if (!ok) {
            // copies that never completed: report, give them one more bounded wait, stop
            if (lane == 0) atomicOr(a.err, SG_ERR_TIMEOUT);
            tc5::mbar_wait(bar, phase ^ 1);
            return;
          }
        }
        T bn[NC], il[LC + 1];
        if (has) {
          if constexpr (TABLE) {
            float f[NC + LC + 1];
            table_interp_at<NC, LC, false>(reinterpret_cast<const float4*>(a_s + lane * SM::CS), tt, a.ti.inv_h, f,
                                           nullptr);
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
        }
        if constexpr (TABLE) __syncwarp();  // every interval read before the a_lm rows overwrite them
        if (has) {
          const T ux = live ? v.x * inv : T(0), uy = live ? v.y * inv : T(0), uz = live ? v.z * inv : T(1);
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
  const size_t smem = FwdSmem<T, NC, LC, TABLE>::bytes();
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

