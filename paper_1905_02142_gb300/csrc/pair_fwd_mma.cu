// Forward pair kernel of the mixed-precision path with the neighbour contraction on tensor
// cores: the expansion coefficients c_nlm of every atom (Sec. II, Eqs. 01/08, summed over
// neighbours, plus the central atom), as in pair_fwd.cuh, with
//   c[n][lm] = sum_pairs b_n(pair) a_lm(pair),  a_lm = 4 pi ilexp_l(z) Y_lm(r_hat),
// computed as a matrix product per (atom, neighbour species) segment: D[tau][n] +=
// A[tau][pair] B[pair][n] with mma.sync m16n8k16 (FP16 operands, FP32 accumulators).
//
//   one warp per atom, the segment's neighbours taken 32 at a time (one per lane):
//     the lane's table interval is bulk-copied from L2 into shared memory and interpolated
//     (b_n and 4 pi ilexp_l, as in pair_fwd.cuh);
//     B: the 32 b rows as FP16 hi / lo in shared memory, read back as mma fragments with
//        ldmatrix.trans (k = pair, 2 k-steps of 16);
//     A: the harmonic recursion runs on the lanes and streams its values in visit order tau
//        (m = 0 column, then (cos, sin) pairs, as the adjoint kernels order them); every 16
//        values go through a double-buffered 32 x 16 shared tile as hi / lo, are read back
//        with ldmatrix.trans and multiplied at once (hi.hi + hi.lo + lo.hi: ~22 bits, the
//        level of FP32), so no lane ever holds or stores the whole a_lm row;
//   at the end of a segment the accumulators are unscaled, staged as c[n][lm] in shared
//   memory (the central-atom term added) and written out with coalesced stores.
//
// Scaling: b and a are multiplied by fixed powers of two (from the table's maxima and
// |Y_lm| <= sqrt((2l + 1) / 4 pi)) that put their largest values near 2^13, far from the
// FP16 overflow and subnormal ranges; D is unscaled exactly at the end.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "soapmath.cuh"
#include "table.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int FM_WARPS = 4;

template <int NC, int LC> struct FmDims {
  static constexpr int LCC = (LC + 1) * (LC + 1);
  static constexpr int TE = (LC + 2) & ~1;         // m = 0 column, padded to an even count
  static constexpr int TN = TE + LC * (LC + 1);    // tau values
  static constexpr int MT = (TN + 15) / 16;        // m16 tiles of tau
  static constexpr int NT = (NC + 7) / 8;          // n8 tiles of n
  static constexpr int CH = 4 * TableDims<NC, LC>::FP;  // floats of one table interval
  static constexpr int CS = CH + 4;                // slot stride: lanes' 16-byte reads in distinct banks
  static constexpr int ROWB = 48;                  // operand row: 16 halves + 16 B (ldmatrix rows in distinct banks)
  static constexpr int TILE = 32 * ROWB;
  static constexpr int SLOTS = 32 * CS * 4;
  static constexpr int OPER = 6 * TILE;            // a hi, a lo (two buffers each), b hi, b lo
  static constexpr int CST = NC * LCC * 4;         // c staging
  static constexpr int WARP_BYTES =
      ((SLOTS > OPER ? (SLOTS > CST ? SLOTS : CST) : (OPER > CST ? OPER : CST)) + 127) / 128 * 128;
  static constexpr size_t bytes() { return (size_t)FM_WARPS * WARP_BYTES + FM_WARPS * 8; }
};

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// hi / lo FP16 parts of two values, packed as half2 words (first value in the low half)
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// 8 values as one 16-byte chunk of an operand row, in the hi and the lo tile
__device__ __forceinline__ void store_chunk8(unsigned char* hi, unsigned char* lo, const float (&v)[8]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split2(v[2 * i], v[2 * i + 1], h[i], l[i]);
  *reinterpret_cast<uint4*>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo) = make_uint4(l[0], l[1], l[2], l[3]);
}

// (l, m) index l^2 + l + m of visit position tau, or -1 for a padding position
template <int LC> __device__ __forceinline__ int lm_of_tau(int tau) {
  constexpr int TE = (LC + 2) & ~1, TN = TE + LC * (LC + 1);
  if (tau < TE) return tau <= LC ? tau * tau + tau : -1;
  if (tau >= TN) return -1;
  const int u = tau - TE;
  int v = u >> 1, m = 1;
  while (v >= LC + 1 - m) {
    v -= LC + 1 - m;
    ++m;
  }
  const int l = m + v;
  return l * l + l + ((u & 1) ? -m : m);
}

template <int NC, int LC>
// 4 blocks per SM (128 registers; a few spills cost less than a quarter of the warps)
__global__ void __launch_bounds__(FM_WARPS * 32, 4) pair_fwd_mma_kernel(const FwdArgs<float> a) {
  using Dm = FmDims<NC, LC>;
  constexpr int MT = Dm::MT, NT = Dm::NT, ROWB = Dm::ROWB, TILE = Dm::TILE, LCC = Dm::LCC;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ short lm_tab[MT * 16];  // (l, m) index of each visit position, -1 for padding
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < MT * 16; t += blockDim.x) lm_tab[t] = (short)lm_of_tau<LC>(t);
  __syncthreads();
  unsigned char* wb = smem_raw + (size_t)warp * Dm::WARP_BYTES;
  float* slots = reinterpret_cast<float*>(wb);
  unsigned char* a_hi = wb;              // [2 buffers] 32 rows of ROWB
  unsigned char* a_lo = wb + 2 * TILE;
  unsigned char* b_hi = wb + 4 * TILE;
  unsigned char* b_lo = wb + 5 * TILE;
  float* cst = reinterpret_cast<float*>(wb);  // [NC][LCC] at the end of a segment
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + (size_t)FM_WARPS * Dm::WARP_BYTES) + warp;
  if (lane == 0) {
    tc5::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t phase = 0;
  // ldmatrix row address of this lane: matrix j = lane / 8, row lane % 8 of it
  const int lj = lane >> 3, lr = lane & 7;
  //   A (tau x pair): matrix j covers tau block j & 1 and pair block j >> 1
  const uint32_t a_off = (uint32_t)(((lj >> 1) * 8 + lr) * ROWB + (lj & 1) * 16);
  //   B (pair x n): matrix j covers pair block j & 1 and n block j >> 1
  const uint32_t b_off = (uint32_t)(((lj & 1) * 8 + lr) * ROWB + (lj >> 1) * 16);
  const uint32_t a_hi_s = tc5::smem_u32(a_hi), a_lo_s = tc5::smem_u32(a_lo);
  const uint32_t b_hi_s = tc5::smem_u32(b_hi), b_lo_s = tc5::smem_u32(b_lo);
  const int L = (a.lmax + 1) * (a.lmax + 1);
  const int nch = a.nsp * a.nmax;
  const float unscale = 1.f / (a.mma_sa * a.mma_sb);  // both powers of two: exact

  for (int atom = blockIdx.x * FM_WARPS + warp; atom < a.n_atoms; atom += gridDim.x * FM_WARPS) {
    const int spc = a.species[atom];
    for (int s = 0; s < a.nsp; ++s) {
      const int beg = a.seg_offs[atom * a.nsp + s];
      const int end = a.seg_offs[atom * a.nsp + s + 1];
      float d[MT][NT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int i = 0; i < 4; ++i) d[mt][nt][i] = 0.f;

      for (int base = beg; base < end; base += 32) {
        const int pidx = base + lane;
        const bool has = pidx < end;
        Vec4<float> v{0.f, 0.f, 0.f, -1.f};
        if (has) v = a.pair_r[a.pair_idx ? a.pair_idx[pidx] : pidx];
        // |r| < 0 marks a pair beyond r_cut in a list built with a skin: no contribution
        const bool live = v.w >= 0.f;
        const float r = live ? v.w : 1.f, inv = 1.f / r;
        // ---- this batch's table intervals into the slots (the previous batch's and
        //      segment's reads of this area ended at the __syncwarp closing them)
        float tt;
        const int k = table_locate(a.ti, r, tt);
        {
          const int cnt = min(32, end - base);
          tc5::fence_proxy_async();
          if (lane == 0) tc5::mbar_expect_tx(bar, (uint32_t)(cnt * Dm::CH * sizeof(float)));
          __syncwarp();
          if (has)
            tc5::bulk_load(slots + lane * Dm::CS, a.table + (size_t)k * (Dm::CH / 2), Dm::CH * sizeof(float), bar);
          const bool ok = __all_sync(0xffffffffu, tc5::mbar_wait(bar, phase));
          phase ^= 1;
          if (!ok) {
            // copies that never completed: report, give them one more bounded wait, stop
            if (lane == 0) atomicOr(a.err, SG_ERR_TIMEOUT);
            tc5::mbar_wait(bar, phase ^ 1);
            return;
          }
        }
        float bv[16], il[LC + 1];
#pragma unroll
        for (int n = 0; n < 16; ++n) bv[n] = 0.f;
#pragma unroll
        for (int l = 0; l <= LC; ++l) il[l] = 0.f;
        if (has && live) {
          float f[NC + LC + 1];
          table_interp_at<NC, LC, false, false, true>(reinterpret_cast<const float4*>(slots + lane * Dm::CS), tt,
                                                      a.ti.inv_h, f, nullptr);
#pragma unroll
          for (int n = 0; n < NC; ++n) bv[n] = f[n] * a.mma_sb;
#pragma unroll
          for (int l = 0; l <= LC; ++l) il[l] = f[NC + l] * a.mma_sa;
        }
        __syncwarp();  // every slot read before the operand tiles overwrite them
        {
          float lo8[8], hi8[8];
#pragma unroll
          for (int n = 0; n < 8; ++n) {
            lo8[n] = bv[n];
            hi8[n] = bv[8 + n];
          }
          store_chunk8(b_hi + lane * ROWB, b_lo + lane * ROWB, lo8);
          store_chunk8(b_hi + lane * ROWB + 16, b_lo + lane * ROWB + 16, hi8);
        }
        // ---- the recursion's values in visit order, 8 at a time into the a tiles; every 16
        //      (one m16 tile) multiplied with the b fragments, which are re-read per tile
        //      (ldmatrix from the b tiles) rather than held in registers
        const float ux = live ? v.x * inv : 0.f, uy = live ? v.y * inv : 0.f, uz = live ? v.z * inv : 1.f;
        float buf[8];
        int tau = 0;
        auto mma_tile = [&](int mt) {
          const int sb = mt & 1;
          __syncwarp();
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            uint32_t ah[4], al[4], bh[4], bl[4];  // b: n tile 0 (b0b1, b2b3), n tile 1 (b0b1, b2b3)
            ldsm_x4_t(a_hi_s + sb * TILE + ks * 16 * ROWB + a_off, ah);
            ldsm_x4_t(a_lo_s + sb * TILE + ks * 16 * ROWB + a_off, al);
            ldsm_x4_t(b_hi_s + ks * 16 * ROWB + b_off, bh);
            ldsm_x4_t(b_lo_s + ks * 16 * ROWB + b_off, bl);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
              mma16816(d[mt][nt], ah, bh[2 * nt], bh[2 * nt + 1]);
              mma16816(d[mt][nt], ah, bl[2 * nt], bl[2 * nt + 1]);
              mma16816(d[mt][nt], al, bh[2 * nt], bh[2 * nt + 1]);
            }
          }
        };
        auto put = [&](float x) {
          buf[tau & 7] = x;
          if ((tau & 7) == 7) {
            const int mt = tau >> 4, half = (tau >> 3) & 1, sb = mt & 1;
            store_chunk8(a_hi + sb * TILE + lane * ROWB + half * 16, a_lo + sb * TILE + lane * ROWB + half * 16, buf);
            if (half) mma_tile(mt);
          }
          ++tau;
        };
        for_each_ylm<float, LC>(ux, uy, uz, a.yc, [&](int l, int m, float y) {
          put(il[l] * y);
          if (m == 0 && l == LC && Dm::TE > LC + 1) put(0.f);  // pad the m = 0 column
        });
        while (tau < MT * 16) put(0.f);
        __syncwarp();  // the last tiles read before the next batch's copies
      }
      // ---- accumulators -> c[n][lm] (unscaled) in shared memory -> global
      const int g = lane >> 2, c2 = (lane & 3) * 2;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int lm0 = lm_tab[16 * mt + g], lm1 = lm_tab[16 * mt + g + 8];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int n = 8 * nt + c2;
          if (lm0 >= 0) {
            if (n < NC) cst[n * LCC + lm0] = d[mt][nt][0] * unscale;
            if (n + 1 < NC) cst[(n + 1) * LCC + lm0] = d[mt][nt][1] * unscale;
          }
          if (lm1 >= 0) {
            if (n < NC) cst[n * LCC + lm1] = d[mt][nt][2] * unscale;
            if (n + 1 < NC) cst[(n + 1) * LCC + lm1] = d[mt][nt][3] * unscale;
          }
        }
      }
      __syncwarp();
      if (s == spc && lane == 0) {
#pragma unroll
        for (int n = 0; n < NC; ++n) cst[n * LCC] += a.bc.cen[n];
      }
      __syncwarp();
      for (int n = 0; n < a.nmax; ++n) {
        float* crow = a.c + ((size_t)atom * nch + s * a.nmax + n) * L;
        for (int lm = lane; lm < L; lm += 32) crow[lm] = cst[n * LCC + lm];
      }
      __syncwarp();  // staging read before the next segment's copies overwrite it
    }
  }
}

template <int NC, int LC>
cudaError_t launch_fwd_mma(const FwdArgs<float>& a, cudaStream_t st) {
  using Dm = FmDims<NC, LC>;
  const size_t smem = Dm::bytes();
  auto kern = pair_fwd_mma_kernel<NC, LC>;
  cudaError_t e = sg_set_smem<pair_fwd_mma_kernel<NC, LC>>(smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FM_WARPS * 32, smem);
  if (per_sm < 1) per_sm = 1;
  long long need = (a.n_atoms + FM_WARPS - 1) / FM_WARPS;
  long long grid = (long long)sms * per_sm * 4;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, FM_WARPS * 32, smem, st>>>(a);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

}  // namespace

bool sg_pair_forward_mma_supported(int cls) { return cls >= 0 && cls <= 3; }

cudaError_t sg_pair_forward_mma(const FwdArgs<float>& a, int cls, cudaStream_t st) {
  if (a.n_atoms == 0) return cudaSuccess;
  if (!(a.mma_sa > 0.f) || !(a.mma_sb > 0.f)) return cudaErrorInvalidValue;
  switch (cls) {
    case 0: return launch_fwd_mma<6, 6>(a, st);
    case 1: return launch_fwd_mma<8, 8>(a, st);
    case 2: return launch_fwd_mma<10, 10>(a, st);
    case 3: return launch_fwd_mma<12, 12>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
