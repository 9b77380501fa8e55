// Adjoint pair kernel of the mixed-precision path on the 5th-generation tensor cores
// (tcgen05, accumulators in tensor memory).  Same mathematics as pair_adj_mma.cu and
// pair_adj.cuh: dE/dq -> dE/dp -> dE/dc (the derivative of Eq. 09) -> dE/dr_ij per pair,
// recomputing the pair's radial terms (Eq. 04 through the radial table) and its real
// harmonics (Sec. III.C) instead of storing dc/dr.
//
//   the G-operand kernel (adj_gop_kernel), one block per atom: h = dE/dp, G_l = M_l c_l,
//     scaled by a power of two and stored as FP16 split rows G16[tau] (B operand, K-major,
//     128-byte swizzled rows; tau = harmonic index in the recursion's visit order) in a
//     per-atom image in global memory, with the exponent of the scale: rows tau and tau + 64
//     of each 128 share one 128-byte row (its first and second 64 bytes) when a split row
//     takes 64 bytes (n_max <= 10), as the A tile packs b and b'
//   the adjoint kernel, one block of 3 warps per atom (persistent over atoms): the atom's
//     image is bulk-copied into one of two shared-memory buffers while the block works on
//     the previous atom; then one thread per pair, 96 pairs of one (atom, neighbour
//     species) segment per tile (the MMA's rows 96..127 are not read), the pair's radial
//     factors in registers for the sweep (168 registers, 4 blocks per SM):
//     b_n(r) and b_n'(r) from the radial table, as FP16 split rows of the A operand
//     u[pair][tau] = sum_n b_n G[tau][n] and u'[pair][tau] = sum_n b_n' G[tau][n]:
//       tcgen05.mma M = 128 pairs, N = 64 harmonics per phase, K = 3 n_max (padded to 16),
//       issued by one thread, FP32 accumulators in 128 TMEM columns (u | u'); TMEM lane =
//       pair, so each thread reads its own pair's u, u' with tcgen05.ld
//     the harmonic sweep of the pair (one thread) consumes 16 harmonics per TMEM read; a
//     block barrier between phases lets the next MMA overwrite the columns
//
// The FP16 split x = hi + lo with the three products hi.hi + hi.lo + lo.hi stacked along k,
// and the power-of-two scalings of G (per atom) and of b, b' (per pair), are those of
// pair_adj_mma.cu: ~22 significant bits, the level of FP32 arithmetic.
// Only exact basis sizes (n_max, l_max equal to the compiled class) take this kernel; the
// sweep is fully unrolled so that every TMEM column index is a compile-time register.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "adj_common.cuh"
#include "internal.h"
#include "table.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int TC_THREADS = 96;         // 3 warps, one pair per thread: 96 of the MMA's 128 rows
constexpr int GOP_THREADS = 128;       // G-operand kernel
constexpr int TC_PHASE = 64;           // harmonics per MMA phase
constexpr uint32_t TC_TMEM_COLS = 128; // u (64 columns) | u' (64 columns)

template <int NC, int LC> struct TcDims {
  static constexpr int KP = (3 * NC + 15) / 16 * 16;  // split operand length (halves)
  static constexpr int KS = KP / 16;                  // MMA k-steps of 16
  static constexpr bool PACKED = KP <= 32;            // b and b' rows share one 128-byte row
  static constexpr int NP = (NC + 3) / 4 * 4;
  static constexpr int LP = LC + 1;
  static constexpr int TE = (LC + 2) & ~1;
  static constexpr int TN = TE + LC * (LC + 1);
  static constexpr int T16 = (TN + 15) & ~15;         // harmonic rows (B operand rows)
  static constexpr int NPH = (T16 + TC_PHASE - 1) / TC_PHASE;
  static constexpr int A_BYTES = PACKED ? 128 * 128 : 2 * 128 * 128;
  // image of one species: with split rows of at most 64 bytes (PACKED), phase ph (harmonic rows
  // 64 ph + [0, 64)) in image rows (ph / 2) 64 + [0, 64), bytes (ph % 2) 64 + [0, 64); else
  // one harmonic row per image row
  static constexpr int ROWS = PACKED ? 64 * ((NPH + 1) / 2) : T16;
  static constexpr int IMG = ROWS * 128;
  __device__ __forceinline__ static int img_row(int tau) { return PACKED ? ((tau >> 6) >> 1) * 64 + (tau & 63) : tau; }
  __device__ __forceinline__ static int img_chunk(int tau) { return PACKED ? ((tau >> 6) & 1) * 4 : 0; }
  // byte offset of phase ph's first row in the image
  __device__ __forceinline__ static uint32_t img_phase(int ph) {
    return PACKED ? (uint32_t)((ph >> 1) * 64 * 128 + (ph & 1) * 64) : (uint32_t)(ph * 64 * 128);
  }
};

struct TcLayout {
  int off_g16;    // two buffers of the atom's image ([nsp][ROWS] rows of 128 B each)
  int off_union;  // the A tile(s)
  int off_red;
  int total;      // bytes to request (includes 1024 for the base alignment)
};

struct GopLayout {
  int off_pc;     // packed channel-pair decode
  int off_scr;    // scratch: dE/dp, q, dE/dq, c, M, G (FP32)
  int off_red;
  int total;
};

// scratch of the G-operand kernel, in floats: [q | dE/dq], later reused for G; c; M
template <int NC, int LC>
int gop_scratch_floats(int nsp, int dim) {
  using Dm = TcDims<NC, LC>;
  const int nch = nsp * NC, L = Dm::LP * Dm::LP;
  return std::max(2 * align4(dim), nsp * Dm::T16 * Dm::NP) + align4(nch * L) + nsp * Dm::LP * nch * Dm::NP;
}

template <int NC, int LC>
TcLayout make_tc_layout(int nsp) {
  using Dm = TcDims<NC, LC>;
  TcLayout m{};
  m.off_g16 = 0;
  m.off_union = (2 * nsp * Dm::IMG + 1023) / 1024 * 1024;
  m.off_red = (m.off_union + Dm::A_BYTES + 15) / 16 * 16;
  m.total = m.off_red + (TC_THREADS / 32 * 9) * 4 + 1024;
  // at most 4 blocks per SM (228 KB of shared memory, 1 KB reserved per block), so that the
  // blocks' tensor-memory allocations (4 x 128 columns) never exceed the SM's 512
  m.total = std::max(m.total, 47 * 1024);
  return m;
}

template <int NC, int LC>
GopLayout make_gop_layout(int nsp, int dim) {
  using Dm = TcDims<NC, LC>;
  GopLayout m{};
  const int nch = nsp * NC;
  m.off_pc = 0;
  m.off_scr = (m.off_pc + 4 * (nch * (nch + 1) / 2) + 15) / 16 * 16;
  m.off_red = m.off_scr + 4 * gop_scratch_floats<NC, LC>(nsp, dim);
  m.total = m.off_red + 4 * 8;
  return m;
}

// FP16 split row in the 128-byte swizzled K-major layout: chunks chunk0 .. chunk0 + KP/8 - 1
// of row `row` hold [hi | hi | lo] (A side) or [hi | lo | hi] (B side), zero-padded to KP.
template <int NC, int KP, bool A_SIDE>
__device__ __forceinline__ void write_split_row_sw(unsigned char* tile, int row, int chunk0,
                                                   const float (&v)[NC]) {
  __half hi[NC], lo[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    hi[n] = __float2half_rn(v[n]);
    lo[n] = __float2half_rn(v[n] - __half2float(hi[n]));
  }
  auto elem = [&](int k) -> __half {
    if (k < NC) return hi[k];
    if (k < 2 * NC) return A_SIDE ? hi[k - NC] : lo[k - NC];
    if (k < 3 * NC) return A_SIDE ? lo[k - 2 * NC] : hi[k - 2 * NC];
    return __ushort_as_half(0);
  };
#pragma unroll
  for (int c = 0; c < KP / 8; ++c) {
    uint4 w;
    w.x = pack_half2(elem(8 * c + 0), elem(8 * c + 1));
    w.y = pack_half2(elem(8 * c + 2), elem(8 * c + 3));
    w.z = pack_half2(elem(8 * c + 4), elem(8 * c + 5));
    w.w = pack_half2(elem(8 * c + 6), elem(8 * c + 7));
    *reinterpret_cast<uint4*>(tile + tc5::sw128_off(row, chunk0 + c)) = w;
  }
}

__device__ __forceinline__ void phase_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(TC_THREADS) : "memory"); }

// The (l, m) sweep of one pair, fully unrolled for l_max = LC (as adj_sweep_unrolled in
// pair_adj_mma.cu), reading u / u' of harmonic tau from ur / upr[tau & 15] after
// refill(tau >> 4) at every multiple of 16.
template <int LC, typename Refill>
__device__ __forceinline__ void tc_sweep(const YlmCoef<float>& yc, float ux, float uy, float uz,
                                         const float (&il_l)[LC + 1], const float (&dil_l)[LC + 1],
                                         const uint32_t (&ur)[16], const uint32_t (&upr)[16], Refill&& refill,
                                         float& srad, float& hx, float& hy, float& hz) {
  constexpr int TE = (LC + 2) & ~1;
  float cm = 1.f, sm = 0.f, cmm1 = 0.f, smm1 = 0.f;
  // column m + 1 of the recursion, computed at step m for the z-derivatives, is column m of
  // step m + 1: kept here (registers, the loops being unrolled) instead of recomputed
  float col[LC + 2];
#pragma unroll
  for (int m = 0; m <= LC; ++m) {
    if (m > 0) {
      cmm1 = cm;
      smm1 = sm;
      cm = ux * cmm1 - uy * smm1;
      sm = ux * smm1 + uy * cmm1;
    }
    float a1 = yc.seed[m], a2 = 0.f;
    float b1 = (m + 1 <= LC) ? yc.seed[m + 1] : 0.f, b2 = 0.f;
    float Rc = 0.f, Rs = 0.f, Xc = 0.f, Xs = 0.f, Zc = 0.f, Zs = 0.f;
#pragma unroll
    for (int l = m; l <= LC; ++l) {
      float pl, ql = 0.f;
      if (m > 0) {
        pl = col[l];
      } else if (l == m) {
        pl = a1;
      } else {
        pl = (l == m + 1) ? (yc.s1[m] * uz) * a1 : fmaf(yc.a[l][m] * uz, a1, -yc.b[l][m] * a2);
        a2 = a1;
        a1 = pl;
      }
      if (m + 1 <= LC && l >= m + 1) {
        if (l == m + 1) {
          ql = b1;
        } else {
          ql = (l == m + 2) ? (yc.s1[m + 1] * uz) * b1 : fmaf(yc.a[l][m + 1] * uz, b1, -yc.b[l][m + 1] * b2);
          b2 = b1;
          b1 = ql;
        }
        col[l] = ql;
      }
      const float dz = yc.d[l][m] * ql;
      const float il = il_l[l], dil = dil_l[l];
      // tau of (l, m): l for m = 0, else the cos-type entry of the (cos, sin) pair
      const int tau = m == 0 ? l : TE + 2 * ((m - 1) * (LC + 1) - m * (m - 1) / 2) + 2 * (l - m);
      if ((tau & 15) == 0) refill(tau >> 4);
      const int k = tau & 15;
      if (m == 0) {
        const float uu = __uint_as_float(ur[k]), up = __uint_as_float(upr[k]);
        Rc = fmaf(fmaf(up, il, uu * dil), pl, Rc);
        Zc = fmaf(uu * il, dz, Zc);
      } else {
        const float uc = __uint_as_float(ur[k]), us = __uint_as_float(ur[k + 1]);
        const float pc = __uint_as_float(upr[k]), ps = __uint_as_float(upr[k + 1]);
        // the radial and harmonic factors shared by the cos- and sin-type entries
        const float e = il * pl, f = dil * pl, g = il * dz;
        Rc = fmaf(pc, e, fmaf(uc, f, Rc));
        Rs = fmaf(ps, e, fmaf(us, f, Rs));
        Xc = fmaf(uc, e, Xc);
        Xs = fmaf(us, e, Xs);
        Zc = fmaf(uc, g, Zc);
        Zs = fmaf(us, g, Zs);
      }
    }
    if (m == 0) {
      srad += Rc;
      hz += Zc;
    } else {
      const float fm = (float)m;
      srad = fmaf(Rc, cm, fmaf(Rs, sm, srad));
      hx = fmaf(fm, fmaf(Xc, cmm1, Xs * smm1), hx);
      hy = fmaf(fm, fmaf(Xs, cmm1, -Xc * smm1), hy);
      hz = fmaf(Zc, cm, fmaf(Zs, sm, hz));
    }
  }
}

// The per-atom G operand of the adjoint (one block per atom, persistent): h = dE/dp, the
// packed-pair derivative matrices M, G = M c in FP32, scaled by 2^(14 - e) with 2^e > max |G|
// and split into FP16 rows, written to the atom's image (each thread 64 bytes of a row: two
// whole 32-byte sectors), and e.
template <int NC, int LC>
__global__ void __launch_bounds__(GOP_THREADS) adj_gop_kernel(const AdjArgs<float> a, const GopLayout lay) {
  using Dm = TcDims<NC, LC>;
  constexpr int KP = Dm::KP, NP = Dm::NP, LP = Dm::LP, T16 = Dm::T16;
  constexpr int TE = Dm::TE, TN = Dm::TN;
  constexpr int W = GOP_THREADS / 32, NT = GOP_THREADS;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  constexpr int lmax = LC, nmax = NC;
  constexpr int L = LP * LP, lp1 = LP;
  const int nch = a.nsp * nmax;
  const int D = a.dim;
  const int npair = nch * (nch + 1) / 2;
  int* pcdec = reinterpret_cast<int*>(smem + lay.off_pc);
  float* qs = reinterpret_cast<float*>(smem + lay.off_scr);  // [D]
  float* gs = qs + align4(D);                                 // [D] dE/dq
  float* g32 = qs;  // [nsp][T16][NP] G (several species), written once q and dE/dq are used up
  float* cs = qs + max(2 * align4(D), a.nsp * T16 * NP);      // [nch][L]
  float* ms = cs + align4(nch * L);                           // [nsp][lp1][nch][NP]
  float* red2 = reinterpret_cast<float*>(smem + lay.off_red);
  const uint32_t img_bytes = (uint32_t)(a.nsp * Dm::IMG);

  for (int pc = tid; pc < npair; pc += NT) {
    int c1 = 0, rem = pc;
    while (rem >= nch - c1) {
      rem -= nch - c1;
      ++c1;
    }
    pcdec[pc] = c1 | ((c1 + rem) << 16);
  }
  __syncthreads();
  for (int atom = blockIdx.x; atom < a.n_atoms; atom += gridDim.x) {
    __syncthreads();  // the previous atom done with the scratch
    // ---- c, q, g -> shared memory: asynchronous copies, all in flight together
    {
      const float* qi = a.q + (size_t)atom * D;
      const float* gi = a.g + (size_t)atom * D;
      const float* ci = a.c + (size_t)atom * nch * L;
      for (int k = tid; k < nch * L; k += NT) cp_async4(cs + k, ci + k);
      for (int k = tid; k < D; k += NT) {
        cp_async4(qs + k, qi + k);
        cp_async4(gs + k, gi + k);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    const float w = (float)a.struct_w[a.atom_struct[atom]];
    const float pn = a.pnorm[atom];
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    // ---- h = dE/dp = w (g - q (q.g)) / |p|, formed where M needs it
    float dot = 0.f;
    for (int k = tid; k < D; k += NT) dot += qs[k] * gs[k];
    dot = block_sum<W>(dot, red2);
    const float sc = w / pn;

    // ---- M[s][l][c2][n] = d p_(c1 c2 l) / d(c1, c2 product) with c1 = (s, n): 2 h on the
    //      diagonal, sqrt(2) h off it; one thread per packed channel pair writes both halves
    for (int pc = tid; pc < npair; pc += NT) {
      const int dec = pcdec[pc];
      const int c1 = dec & 0xffff, c2 = dec >> 16;
      const int s1 = c1 / nmax, n1 = c1 - s1 * nmax;
      const int s2 = c2 / nmax, n2 = c2 - s2 * nmax;
      const float f = c1 == c2 ? 2.f : 1.41421356237f;
      const float* qrow = qs + pc * lp1;
      const float* grow = gs + pc * lp1;
      float* m1 = ms + ((size_t)s1 * lp1 * nch + c2) * NP + n1;  // + l nch NP
      float* m2 = ms + ((size_t)s2 * lp1 * nch + c1) * NP + n2;
      for (int l = 0; l <= lmax; ++l) {
        const float hv = f * (sc * (grow[l] - qrow[l] * dot));
        m1[(size_t)l * nch * NP] = hv;
        if (c1 != c2) m2[(size_t)l * nch * NP] = hv;
      }
    }
    __syncthreads();

    // ---- G[s][lm][n] = sum_c2 M[s][l][c2][n] c[c2][lm], one thread per lm row
    auto grow_of = [&](int lm, int l, int sp, float (&acc)[NP]) {
#pragma unroll
      for (int n = 0; n < NP; ++n) acc[n] = 0.f;
      const float4* m4 = reinterpret_cast<const float4*>(ms + (size_t)(sp * lp1 + l) * nch * NP);
      const float* cp = cs + lm;
#pragma unroll 2
      for (int c2 = 0; c2 < nch; ++c2) {
        const float cv = cp[c2 * L];
#pragma unroll
        for (int q4 = 0; q4 < NP / 4; ++q4) {
          const float4 mv = m4[c2 * (NP / 4) + q4];
          if (4 * q4 + 0 < NC) acc[4 * q4 + 0] = fmaf(mv.x, cv, acc[4 * q4 + 0]);
          if (4 * q4 + 1 < NC) acc[4 * q4 + 1] = fmaf(mv.y, cv, acc[4 * q4 + 1]);
          if (4 * q4 + 2 < NC) acc[4 * q4 + 2] = fmaf(mv.z, cv, acc[4 * q4 + 2]);
          if (4 * q4 + 3 < NC) acc[4 * q4 + 3] = fmaf(mv.w, cv, acc[4 * q4 + 3]);
        }
      }
    };
    unsigned char* img = a.gimg + (size_t)atom * img_bytes;
    float gmax = 0.f;
    int eg = 0;
    if (a.nsp == 1) {
      // rows kept in registers across the block maximum, then scaled, split and written; the
      // padding rows of the image are never read by the adjoint's sweep and stay unwritten
      constexpr int RPT = (L + NT - 1) / NT;
      float accr[RPT][NP];
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int lm = tid + r * NT;
        if (lm < L) {
          grow_of(lm, (int)sqrtf((float)lm + 0.5f), 0, accr[r]);
#pragma unroll
          for (int n = 0; n < NC; ++n) gmax = fmaxf(gmax, fabsf(accr[r][n]));
        }
      }
      gmax = block_max<W>(gmax, red2 + W);
      frexpf(gmax, &eg);
      eg = max(-100, min(eg, 100));
      const float sg = ldexpf(1.f, 14 - eg);
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int lm = tid + r * NT;
        if (lm < L) {
          const int l = (int)sqrtf((float)lm + 0.5f);
          const int tau = tau_of(l, lm - l * l - l, lmax);
          float v[NC];
#pragma unroll
          for (int n = 0; n < NC; ++n) v[n] = accr[r][n] * sg;
          write_split_row_sw<NC, KP, false>(img, Dm::img_row(tau), Dm::img_chunk(tau), v);
        }
      }
    } else {
      for (int lm = tid; lm < L; lm += NT) {
        const int l = (int)sqrtf((float)lm + 0.5f);
        const int tau = tau_of(l, lm - l * l - l, lmax);
        for (int sp = 0; sp < a.nsp; ++sp) {
          float acc[NP];
          grow_of(lm, l, sp, acc);
#pragma unroll
          for (int n = 0; n < NP; ++n) {
            if (!(n < NC)) acc[n] = 0.f;
            gmax = fmaxf(gmax, fabsf(acc[n]));
          }
          float4* row = reinterpret_cast<float4*>(g32 + ((size_t)sp * T16 + tau) * NP);
#pragma unroll
          for (int q4 = 0; q4 < NP / 4; ++q4)
            row[q4] = make_float4(acc[4 * q4], acc[4 * q4 + 1], acc[4 * q4 + 2], acc[4 * q4 + 3]);
        }
      }
      gmax = block_max<W>(gmax, red2 + W);
      frexpf(gmax, &eg);
      eg = max(-100, min(eg, 100));
      const float sg = ldexpf(1.f, 14 - eg);
      for (int row = tid; row < a.nsp * T16; row += NT) {
        const int sp = row / T16, tau = row - sp * T16;
        const bool real = tau < TE ? tau <= lmax : tau < TN;
        float v[NC];
        const float4* r4 = reinterpret_cast<const float4*>(g32 + (size_t)row * NP);
#pragma unroll
        for (int q4 = 0; q4 < NP / 4; ++q4) {
          const float4 x = real ? r4[q4] : make_float4(0.f, 0.f, 0.f, 0.f);
          if (4 * q4 + 0 < NC) v[4 * q4 + 0] = x.x * sg;
          if (4 * q4 + 1 < NC) v[4 * q4 + 1] = x.y * sg;
          if (4 * q4 + 2 < NC) v[4 * q4 + 2] = x.z * sg;
          if (4 * q4 + 3 < NC) v[4 * q4 + 3] = x.w * sg;
        }
        write_split_row_sw<NC, KP, false>(img + (size_t)sp * Dm::IMG, Dm::img_row(tau), Dm::img_chunk(tau), v);
      }
    }
    if (tid == 0) a.gexp[atom] = eg;
  }
}

template <int NC, int LC>
__global__ void __launch_bounds__(TC_THREADS, 4) pair_adj_tc_kernel(const AdjArgs<float> a, const TcLayout lay) {
  using Dm = TcDims<NC, LC>;
  constexpr int KP = Dm::KP, KS = Dm::KS, LP = Dm::LP, T16 = Dm::T16, NPH = Dm::NPH;
  constexpr int W = TC_THREADS / 32, NT = TC_THREADS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ __align__(8) uint64_t gbar[2];  // per image buffer: its bulk copy has landed
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  unsigned char* gimg = smem + lay.off_g16;  // [2][nsp][ROWS][128 B]
  unsigned char* uni = smem + lay.off_union;
  float* red = reinterpret_cast<float*>(smem + lay.off_red);  // [W][9] virial
  unsigned char* atile = uni;                    // A: b rows (and b' rows when packed)
  unsigned char* atile_p = Dm::PACKED ? uni : uni + 128 * 128;
  constexpr int chunk_p = Dm::PACKED ? 4 : 0;    // first 16-byte chunk of the b' rows

  const uint32_t img_bytes = (uint32_t)(a.nsp * Dm::IMG);
  if (tid == 0) {
    tc5::mbar_init(&mma_bar, 1);
    tc5::mbar_init(&gbar[0], 1);
    tc5::mbar_init(&gbar[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc5::tmem_alloc(&tmem_slot, TC_TMEM_COLS);
  tc5::fence_before();
  __syncthreads();
  tc5::fence_after();
  const uint32_t tmem = tmem_slot;
  uint32_t mma_done = 0;  // MMA phases committed so far (the same count in every thread)
  int buf = 0;            // image buffer of the current atom
  uint32_t gpar = 0;      // bit b: parity of the next completion of gbar[b]
  uint32_t pend = 0;      // (thread 0) bit b: a copy into buffer b not yet waited for
  if (tid == 0 && (int)blockIdx.x < a.n_atoms) {
    tc5::mbar_expect_tx(&gbar[0], img_bytes);
    tc5::bulk_load(gimg, a.gimg + (size_t)blockIdx.x * img_bytes, img_bytes, &gbar[0]);
    pend = 1u;
  }

  for (int atom = blockIdx.x; atom < a.n_atoms; atom += gridDim.x) {
    __syncthreads();  // previous atom done with its image buffer and the A tiles
    // ---- the next atom's image into the other buffer (the previous atom, which used it,
    //      has awaited all its MMAs); then this atom's, copied during the previous atom
    const int nxt = atom + gridDim.x;
    if (tid == 0 && nxt < a.n_atoms && !abort_flag) {
      const int nb = buf ^ 1;
      tc5::mbar_expect_tx(&gbar[nb], img_bytes);
      tc5::bulk_load(gimg + (size_t)nb * img_bytes, a.gimg + (size_t)nxt * img_bytes, img_bytes, &gbar[nb]);
      pend |= 1u << nb;
    }
    if (!abort_flag) {
      if (!tc5::mbar_wait(&gbar[buf], (gpar >> buf) & 1u)) {
        abort_flag = 1;
        if (a.err) atomicOr(a.err, SG_ERR_TIMEOUT);
      } else {
        gpar ^= 1u << buf;
        pend &= ~(1u << buf);
      }
    }
    const int eg = a.gexp[atom];
    __syncthreads();  // every thread past the wait: the image is in shared memory

    // next atom's pair vectors towards L2 while this one's pairs run
    if (nxt < a.n_atoms) {
      const int pb = a.list_offs[nxt * a.nsp], pe = a.list_offs[(nxt + 1) * a.nsp];
      const char* pr = reinterpret_cast<const char*>(a.pair_r + pb);
      const int lp = pe > pb ? (int)(((pe - pb) * sizeof(Vec4<float>) + 127) >> 7) : 0;
      for (int k = tid; k < lp; k += NT) asm volatile("prefetch.global.L2 [%0];" ::"l"(pr + ((size_t)k << 7)));
    }

    float vir[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) vir[t] = 0.f;
    for (int s = 0; s < a.nsp; ++s) {
      const int beg = a.seg_offs[atom * a.nsp + s];
      const int end = a.seg_offs[atom * a.nsp + s + 1];
      const uint32_t gsp = tc5::smem_u32(gimg + (size_t)buf * img_bytes + (size_t)s * Dm::IMG);
      for (int tbase = beg; tbase < end; tbase += NT) {
        // ---- radial terms of this thread's pair -> A rows (b, b'), il and dil (registers)
        const int pidx = tbase + tid;
        const bool valid = pidx < end;
        float ux = 0.f, uy = 0.f, uz = 1.f, r = 1.f, inv_r = 1.f;
        Vec4<float> v{};
        const int pp = (valid && a.pair_idx) ? a.pair_idx[pidx] : pidx;  // index in the full list
        if (valid) v = a.pair_r[pp];
        // |r| < 0 marks a pair beyond r_cut in a list built with a skin: dE/dr = 0
        const bool live = valid && v.w >= 0.f;
        if (live) {
          r = v.w;
          inv_r = 1.f / r;
          ux = v.x * inv_r;
          uy = v.y * inv_r;
          uz = v.z * inv_r;
        }
        int eb = 0;
        float il[LP], dil[LP];  // 4 pi ilexp_l and its r-derivative, kept for the sweep
        {
          float f[NC + LC + 1], df[NC + LC + 1];
          table_interp<NC, LC, true>(a.table, a.ti, r, f, df);
          float bn[NC], dbn[NC];
          float bmax = 0.f;
#pragma unroll
          for (int n = 0; n < NC; ++n) {
            bn[n] = live ? f[n] : 0.f;
            dbn[n] = live ? df[n] : 0.f;
            bmax = fmaxf(bmax, fmaxf(fabsf(bn[n]), fabsf(dbn[n])));
          }
          frexpf(bmax, &eb);
          eb = max(-100, min(eb, 100));
          const float sb = ldexpf(1.f, 14 - eb);
#pragma unroll
          for (int n = 0; n < NC; ++n) {
            bn[n] *= sb;
            dbn[n] *= sb;
          }
          write_split_row_sw<NC, KP, true>(atile, tid, 0, bn);
          write_split_row_sw<NC, KP, true>(atile_p, tid, chunk_p, dbn);
#pragma unroll
          for (int l = 0; l < LP; ++l) {
            il[l] = f[NC + l];
            dil[l] = df[NC + l];
          }
        }
        tc5::fence_proxy_async();  // the A rows, written by threads, reach the tensor cores
        __syncthreads();

        // ---- phases: u, u' of 64 harmonics at a time in TMEM, consumed by the sweep
        auto issue = [&](int ph) {
          const int n = min(TC_PHASE, T16 - ph * TC_PHASE);
          const uint32_t idesc = tc5::idesc_f16(128, n);
          const uint32_t a0 = tc5::smem_u32(atile), ap = tc5::smem_u32(atile_p) + chunk_p * 16;
          const uint32_t b0 = gsp + Dm::img_phase(ph);
#pragma unroll
          for (int ks = 0; ks < KS; ++ks) {
            tc5::mma_f16(tmem, tc5::sw128_desc(a0 + ks * 32), tc5::sw128_desc(b0 + ks * 32), idesc, ks > 0);
            tc5::mma_f16(tmem + TC_PHASE, tc5::sw128_desc(ap + ks * 32), tc5::sw128_desc(b0 + ks * 32), idesc,
                         ks > 0);
          }
          tc5::mma_commit(&mma_bar);
        };
        auto await = [&]() {
          if (!abort_flag && !tc5::mbar_wait(&mma_bar, mma_done & 1)) {
            abort_flag = 1;
            if (a.err) atomicOr(a.err, SG_ERR_TIMEOUT);
          }
          ++mma_done;
          __syncwarp();  // the lanes leave the wait loop at different times
          tc5::fence_after();
        };
        const bool wactive = tbase + warp * 32 < end;  // this warp holds at least one pair
        float srad = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
        if (wactive) {
          uint32_t ur[16], upr[16];
          auto refill = [&](int chunk) {
            if ((chunk & 3) == 0) {  // first 16 harmonics of a phase
              const int ph = chunk >> 2;
              if (ph > 0) {
                tc5::fence_before();
                phase_barrier();  // every warp has read the previous phase's columns
              }
              if (tid == 0) {
                tc5::fence_after();
                issue(ph);
              }
              await();
            }
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((chunk & 3) * 16);
            tc5::tmem_ld16_nw(ta, ur);
            tc5::tmem_ld16_nw(ta + TC_PHASE, upr);
            tc5::tmem_wait();
          };
          tc_sweep<LC>(a.yc, ux, uy, uz, il, dil, ur, upr, refill, srad, hx, hy, hz);
        } else {
          // no pair in this warp: only the phase barriers, and the MMA counter
          for (int ph = 0; ph < NPH; ++ph) {
            if (ph > 0) phase_barrier();
            ++mma_done;
          }
        }
        if (valid && !live) a.dedr[pp] = Vec4<float>{0.f, 0.f, 0.f, 0.f};
        if (live) {
          const float inv_s = ldexpf(1.f, eg + eb - 28);
          srad *= inv_s;
          hx *= inv_s;
          hy *= inv_s;
          hz *= inv_s;
          const float hdot = hx * ux + hy * uy + hz * uz;
          Vec4<float> o;
          o.x = ux * srad + (hx - hdot * ux) * inv_r;
          o.y = uy * srad + (hy - hdot * uy) * inv_r;
          o.z = uz * srad + (hz - hdot * uz) * inv_r;
          o.w = 0.f;
          a.dedr[pp] = o;
          const float gv[3] = {o.x, o.y, o.z}, rv[3] = {v.x, v.y, v.z};
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) vir[3 * p + q2] -= gv[p] * rv[q2];
        }
        tc5::fence_before();
        __syncthreads();  // tensor memory and the A tiles free for the next tile
      }
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const float vt = warp_sum(vir[t]);
      if (lane == 0) red[warp * 9 + t] = vt;
    }
    __syncthreads();
    if (tid < 9) {
      float vt = 0.f;
#pragma unroll
      for (int w2 = 0; w2 < W; ++w2) vt += red[w2 * 9 + tid];
      a.vir_atom[(size_t)atom * 9 + tid] = vt;
    }
    buf ^= 1;
  }
  // after a timeout the block stopped waiting: give a copy still in flight one more bounded
  // wait before the shared memory is released
  if (tid == 0 && abort_flag)
    for (int b = 0; b < 2; ++b)
      if (pend & (1u << b)) tc5::mbar_wait(&gbar[b], (gpar >> b) & 1u);
  tc5::fence_before();
  __syncthreads();
  if (warp == 0) tc5::tmem_dealloc(tmem, TC_TMEM_COLS);
}

template <int NC, int LC>
cudaError_t launch_tc(const AdjArgs<float>& a, cudaStream_t st) {
  if (!a.gimg || !a.gexp) return cudaErrorInvalidValue;
  int dev = 0, sms = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    return cudaGetLastError();
  // ---- the per-atom G operand images
  const GopLayout gl = make_gop_layout<NC, LC>(a.nsp, a.dim);
  if (gl.total > 220 * 1024) return cudaErrorInvalidConfiguration;
  {
    auto kern = adj_gop_kernel<NC, LC>;
    cudaError_t e = sg_set_smem<adj_gop_kernel<NC, LC>>(gl.total);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GOP_THREADS, gl.total);
    long long grid = (long long)sms * std::max(1, per_sm);
    if (grid > a.n_atoms) grid = a.n_atoms;
    kern<<<(unsigned)grid, GOP_THREADS, gl.total, st>>>(a, gl);
    ++sg_kernel_launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // ---- the adjoint
  const TcLayout lay = make_tc_layout<NC, LC>(a.nsp);
  if (lay.total > 220 * 1024) return cudaErrorInvalidConfiguration;
  auto kern = pair_adj_tc_kernel<NC, LC>;
  cudaError_t e = sg_set_smem<pair_adj_tc_kernel<NC, LC>>(lay.total);
  if (e != cudaSuccess) return e;
  // resident blocks per SM from the kernel's shared memory and registers (the occupancy
  // query reports one block per SM for kernels that allocate tensor memory), and at most
  // 512 / 128 by the tensor memory
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return cudaGetLastError();
  const int by_smem = smem_sm / (lay.total + (int)fa.sharedSizeBytes + 1024);
  const int by_regs = fa.numRegs > 0 ? 65536 / (((fa.numRegs + 7) & ~7) * TC_THREADS) : 1;
  const int per_sm = std::max(1, std::min(std::min(by_smem, by_regs), (int)(512 / TC_TMEM_COLS)));
  long long grid = (long long)sms * per_sm;
  if (grid > a.n_atoms) grid = a.n_atoms;
  kern<<<(unsigned)grid, TC_THREADS, lay.total, st>>>(a, lay);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

}  // namespace

bool sg_pair_adjoint_tc_supported(const AdjArgs<float>& a, int cls) {
  const int c = cls < 0 ? 0 : (cls > 3 ? 3 : cls);
  return a.nmax == 6 + 2 * c && a.lmax == 6 + 2 * c;
}

cudaError_t sg_pair_adjoint_tc(const AdjArgs<float>& a, int cls, cudaStream_t st) {
  if (a.n_atoms == 0) return cudaSuccess;
  if (!sg_pair_adjoint_tc_supported(a, cls)) return cudaErrorInvalidValue;
  switch (cls) {
    case 0: return launch_tc<6, 6>(a, st);
    case 1: return launch_tc<8, 8>(a, st);
    case 2: return launch_tc<10, 10>(a, st);
    default: return launch_tc<12, 12>(a, st);
  }
}

size_t sg_adj_tc_image_bytes(int cls, int nsp) {
  switch (cls) {
    case 0: return (size_t)nsp * TcDims<6, 6>::IMG;
    case 1: return (size_t)nsp * TcDims<8, 8>::IMG;
    case 2: return (size_t)nsp * TcDims<10, 10>::IMG;
    default: return (size_t)nsp * TcDims<12, 12>::IMG;
  }
}
