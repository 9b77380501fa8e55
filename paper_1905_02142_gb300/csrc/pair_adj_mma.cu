// Adjoint pair kernel of the mixed-precision path with the per-atom contraction on tensor
// cores.  Same mathematics as pair_adj.cuh (dE/dq -> dE/dp -> dE/dc -> dE/dr_ij per pair,
// recomputing the pair's radial and angular terms), organised as:
//
//   one block (4 warps) per atom
//     prologue (128 threads): h = dE/dp, G_l = M_l c_l (derivative of Eq. 09), stored as
//     FP16 hi/lo rows G16[tau][k] after a power-of-two scaling (tau = harmonic index in the
//     order the recursion visits it, see tau_of)
//   one warp per batch of 32 pairs of that atom
//     u[pair][tau]  = sum_n b_n(r) G[tau][n],   u'[pair][tau] = sum_n b_n'(r) G[tau][n]
//       on tensor cores (mma.sync m16n8k16, FP32 accumulate), 16 tau rows at a time;
//       the split x = hi + lo (both FP16) with the three products hi.hi + hi.lo + lo.hi
//       stacked along k keeps ~22 significant bits, the level of FP32 arithmetic
//     dE/dr from u, u' and the harmonic recursion (one lane per pair), as in pair_adj.cuh
//
// Scaling: G is scaled per atom and (b, b') per pair by powers of two so that the largest
// magnitude sits at 2^13..2^14, well inside the FP16 range; the factor is removed from the
// pair's result at the end (exact).
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "adj_common.cuh"
#include "internal.h"
#include "table.cuh"

namespace {


// FP16 operand rows of KP halfs.  KP = 32: 64-byte rows with the 16-byte chunk index XORed
// by (row / 2) % 4, so that the 8 rows an ldmatrix reads hit 8 distinct bank groups.
// KP = 48: 112-byte rows (an odd number of 16-byte chunks) without swizzle.
template <int KP> struct RowLayout {
  static constexpr int kBytes = KP == 32 ? 64 : KP * 2 + 16;
  __device__ __forceinline__ static int off(int row, int chunk) {
    if constexpr (KP == 32) return row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4);
    else return row * kBytes + (chunk << 4);
  }
};


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}


__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                        uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}


// Operand row for a value vector v[0..NC): k = [hi(v) | hi(v) | lo(v) | 0...] (A side) or
// [hi(v) | lo(v) | hi(v) | 0...] (B side), so that the k-sum gives hi.hi + hi.lo + lo.hi.
template <int NC, int KP, bool A_SIDE>
__device__ __forceinline__ void write_split_row(unsigned char* base, int row, const float (&v)[NC]) {
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
    *reinterpret_cast<uint4*>(base + RowLayout<KP>::off(row, c)) = w;
  }
}

struct MmaLayout {
  int t16;        // tau rows per species (multiple of 16)
  int off_g16;    // byte offsets in dynamic shared memory
  int off_union;
  int off_red;
  int loop_warp;  // bytes of one warp's pair-loop scratch
  int total;
};

template <int NC, int LC> struct Dims {
  static constexpr int KP = (3 * NC + 15) / 16 * 16;
  static constexpr int KS = KP / 16;
  static constexpr int RB = RowLayout<KP>::kBytes;
  static constexpr int LP = LC + 1;
  static constexpr int NP = (NC + 3) / 4 * 4;
};

// prologue scratch (floats, each part 16-byte aligned):
//   h [D] | q [D] | g [D] | c [nch][L] | M [nsp][l_max+1][nch][NP] | G [nsp][t16][NP]

template <int NC, int LC>
int prologue_floats(int nsp, int nmax, int lmax, int dim, int t16) {
  const int nch = nsp * nmax, L = (lmax + 1) * (lmax + 1);
  constexpr int NP = Dims<NC, LC>::NP;
  return 3 * align4(dim) + align4(nch * L) + nsp * (lmax + 1) * nch * NP + nsp * t16 * NP;
}

template <int NC, int LC, int W>
MmaLayout make_layout(int nsp, int nmax, int lmax, int dim) {
  using Dm = Dims<NC, LC>;
  MmaLayout m{};
  m.t16 = tau_rows16(lmax);
  const int nch = nsp * nmax;
  const int coef = (int)sizeof(CoefShared<LC>) + 4 * align4(nch * (nch + 1) / 2);
  const int g16 = nsp * m.t16 * Dm::RB;
  const int prologue = 4 * prologue_floats<NC, LC>(nsp, nmax, lmax, dim, m.t16);
  m.loop_warp = 2 * 32 * Dm::RB + 8 * 32 * 16 + 2 * Dm::LP * 32 * 4;
  const int uni = std::max(prologue, W * m.loop_warp);
  m.off_g16 = (coef + 127) / 128 * 128;
  m.off_union = (m.off_g16 + g16 + 127) / 128 * 128;
  m.off_red = (m.off_union + uni + 15) / 16 * 16;
  m.total = m.off_red + (W * 11) * 4;
  return m;
}


// The (l, m) sweep of one pair with l_max = LC known at compile time: fully unrolled, so the
// recursion coefficients are constant-bank operands of the kernel's parameters, every
// shared-memory offset is an immediate, and the 16-row refills of u / u' sit at fixed
// points.  Same arithmetic as the rolled sweep in the kernel (real-harmonic recursion in
// l for columns m and m + 1, cos/sin(m phi) rho^m by rotation).
//   ubx[k]: this lane's entry of ubuf row 0 under column swizzle XOR 2k (see refill)
//   il_l:   this lane's 4 pi ilexp_l at il_l[32 l], its r-derivative at il_l[32 (LP + l)]
template <int LC, typename Refill>
__device__ __forceinline__ void adj_sweep_unrolled(const YlmCoef<float>& yc, float ux, float uy, float uz,
                                                   const float* il_l, const float4* const (&ubx)[4],
                                                   Refill&& refill, float& srad, float& hx, float& hy,
                                                   float& hz) {
  constexpr int LP = LC + 1;
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
      const float il = il_l[32 * l], dil = il_l[32 * (LP + l)];
      // tau of (l, m): l for m = 0, else the cos-type entry of the (cos, sin) pair
      const int tau = m == 0 ? l : TE + 2 * ((m - 1) * (LC + 1) - m * (m - 1) / 2) + 2 * (l - m);
      if ((tau & 15) == 0) refill(tau >> 4);
      const float4 u = ubx[(tau & 6) >> 1][((tau >> 1) & 7) * 32];
      if (m == 0) {
        const float uu = (tau & 1) ? u.z : u.x, up = (tau & 1) ? u.w : u.y;
        Rc = fmaf(fmaf(up, il, uu * dil), pl, Rc);
        Zc = fmaf(uu * il, dz, Zc);
      } else {
        const float wc = u.x * il, ws = u.z * il;
        Rc = fmaf(fmaf(u.y, il, u.x * dil), pl, Rc);
        Rs = fmaf(fmaf(u.w, il, u.z * dil), pl, Rs);
        Xc = fmaf(wc, pl, Xc);
        Xs = fmaf(ws, pl, Xs);
        Zc = fmaf(wc, dz, Zc);
        Zs = fmaf(ws, dz, Zs);
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

template <int NC, int LC, int W, bool EXACT>
__global__ void __launch_bounds__(W * 32, (W == 4 ? 4 : (W == 3 ? 5 : 8)))
pair_adj_mma_kernel(const AdjArgs<float> a, const MmaLayout lay) {
  using Dm = Dims<NC, LC>;
  constexpr int KP = Dm::KP, KS = Dm::KS, RB = Dm::RB, LP = Dm::LP, NP = Dm::NP;
  constexpr int NT = W * 32;
  using RL = RowLayout<KP>;
  extern __shared__ __align__(128) unsigned char smem[];
  CoefShared<LC>& cf = *reinterpret_cast<CoefShared<LC>*>(smem);
  unsigned char* g16 = smem + lay.off_g16;
  unsigned char* uni = smem + lay.off_union;
  float* red = reinterpret_cast<float*>(smem + lay.off_red);  // [W][9] virial | [2 W] reductions
  float* red2 = red + W * 9;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lmax = EXACT ? LC : a.lmax;
  const int nmax = EXACT ? NC : a.nmax;
  const int L = (lmax + 1) * (lmax + 1);
  const int lp1 = lmax + 1;
  const int nch = a.nsp * nmax;
  const int D = a.dim;
  const int t16 = lay.t16;
  const int tE = tau_even(lmax), tN = tau_count(lmax);

  const int npair = nch * (nch + 1) / 2;
  // channel-pair decode table (c1 | c2 << 16 for packed index pc), after the coefficients
  int* pcdec = reinterpret_cast<int*>(smem + sizeof(CoefShared<LC>));
  // prologue scratch (aliases the pair-loop scratch)
  float* hs = reinterpret_cast<float*>(uni);     // [D] dE/dp
  float* qs = hs + align4(D);                    // [D]
  float* gs = qs + align4(D);                    // [D]
  float* cs = gs + align4(D);                    // [nch][L]
  float* ms = cs + align4(nch * L);              // [nsp][lp1][nch][NP]
  float* g32 = ms + a.nsp * lp1 * nch * NP;      // [nsp][t16][NP]
  // pair-loop scratch of this warp
  unsigned char* wbase = uni + (size_t)warp * lay.loop_warp;
  unsigned char* bv = wbase;                                                   // [2][32] rows
  float4* ubuf = reinterpret_cast<float4*>(wbase + 2 * 32 * RB);               // [8][32]
  float* ild = reinterpret_cast<float*>(wbase + 2 * 32 * RB + 8 * 32 * 16);    // [2][LP][32]

  for (int k = tid; k < LP * LP; k += NT) {
    const int l = k / LP, m = k - l * LP;
    cf.p[l][m] = make_float4(coef_a(a.yc, l, m), coef_b(a.yc, l, m), coef_a(a.yc, l, m + 1),
                             coef_b(a.yc, l, m + 1));
    cf.q[l][m] = make_float4(coef_c(a.yc, l, m), coef_c(a.yc, l, m + 1), a.yc.d[l][m], 0.f);
  }
  for (int pc = tid; pc < npair; pc += NT) {
    int c1 = 0, rem = pc;
    while (rem >= nch - c1) {
      rem -= nch - c1;
      ++c1;
    }
    pcdec[pc] = c1 | ((c1 + rem) << 16);
  }

  for (int atom = blockIdx.x; atom < a.n_atoms; atom += gridDim.x) {
    __syncthreads();  // previous atom done with G16 and the scratch; tables visible
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
    // ---- h = dE/dp = w (g - q (q.g)) / |p|
    float dot = 0.f;
    for (int k = tid; k < D; k += NT) dot += qs[k] * gs[k];
    dot = block_sum<W>(dot, red2);
    const float sc = w / pn;
    for (int k = tid; k < D; k += NT) hs[k] = sc * (gs[k] - qs[k] * dot);
    __syncthreads();

    // ---- M[s][l][c2][n] = d p_(c1 c2 l) / d(c1, c2 product) with c1 = (s, n): 2 h on the
    //      diagonal, sqrt(2) h off it; one thread per packed channel pair writes both halves
    for (int pc = tid; pc < npair; pc += NT) {
      const int dec = pcdec[pc];
      const int c1 = dec & 0xffff, c2 = dec >> 16;
      const int s1 = c1 / nmax, n1 = c1 - s1 * nmax;
      const int s2 = c2 / nmax, n2 = c2 - s2 * nmax;
      const float f = c1 == c2 ? 2.f : 1.41421356237f;
      const float* hrow = hs + pc * lp1;
      float* m1 = ms + ((size_t)s1 * lp1 * nch + c2) * NP + n1;  // + l nch NP
      float* m2 = ms + ((size_t)s2 * lp1 * nch + c1) * NP + n2;
      for (int l = 0; l <= lmax; ++l) {
        const float hv = f * hrow[l];
        m1[(size_t)l * nch * NP] = hv;
        if (c1 != c2) m2[(size_t)l * nch * NP] = hv;
      }
    }
    __syncthreads();

    // ---- G[s][lm][n] = sum_c2 M[s][l][c2][n] c[c2][lm]  (n < NC; n >= n_max zeroed below)
    float gmax = 0.f;
    for (int lm = tid; lm < L; lm += NT) {
      const int l = (int)sqrtf((float)lm + 0.5f);
      const int tau = tau_of(l, lm - l * l - l, lmax);
      for (int s = 0; s < a.nsp; ++s) {
        float acc[NP];
#pragma unroll
        for (int n = 0; n < NP; ++n) acc[n] = 0.f;
        const float4* m4 = reinterpret_cast<const float4*>(ms + (size_t)(s * lp1 + l) * nch * NP);
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
#pragma unroll
        for (int n = 0; n < NP; ++n) {
          if (!(n < NC && (EXACT || n < nmax))) acc[n] = 0.f;
          gmax = fmaxf(gmax, fabsf(acc[n]));
        }
        float4* row = reinterpret_cast<float4*>(g32 + ((size_t)s * t16 + tau) * NP);
#pragma unroll
        for (int q4 = 0; q4 < NP / 4; ++q4)
          row[q4] = make_float4(acc[4 * q4], acc[4 * q4 + 1], acc[4 * q4 + 2], acc[4 * q4 + 3]);
      }
    }
    gmax = block_max<W>(gmax, red2 + W);
    int eg = 0;
    frexpf(gmax, &eg);
    eg = max(-100, min(eg, 100));
    const float sg = ldexpf(1.f, 14 - eg);
    for (int row = tid; row < a.nsp * t16; row += NT) {
      const int s = row / t16, tau = row - s * t16;
      const bool real = tau < tE ? tau <= lmax : tau < tN;
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
      write_split_row<NC, KP, false>(g16 + (size_t)s * t16 * RB, tau, v);
    }
    __syncthreads();

    // next atom's inputs towards L2 while this one's pairs run
    {
      const int nxt = atom + gridDim.x;
      if (nxt < a.n_atoms) {
        const int lc = (nch * L * 4 + 127) >> 7, lq = (D * 4 + 127) >> 7;
        const int pb = a.list_offs[nxt * a.nsp], pe = a.list_offs[(nxt + 1) * a.nsp];
        const char* pr = reinterpret_cast<const char*>(a.pair_r + pb);
        const int lp = pe > pb ? (int)(((pe - pb) * sizeof(Vec4<float>) + 127) >> 7) : 0;
        for (int k = tid; k < lc + 2 * lq + lp; k += NT) {
          const char* p;
          if (k < lc) p = reinterpret_cast<const char*>(a.c + (size_t)nxt * nch * L) + ((size_t)k << 7);
          else if (k < lc + lq) p = reinterpret_cast<const char*>(a.q + (size_t)nxt * D) + ((size_t)(k - lc) << 7);
          else if (k < lc + 2 * lq) p = reinterpret_cast<const char*>(a.g + (size_t)nxt * D) + ((size_t)(k - lc - lq) << 7);
          else p = pr + ((size_t)(k - lc - 2 * lq) << 7);
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
        }
      }
    }

    // ---- pair batches: warp w takes batches w, w + W, ... of this atom
    float vir[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) vir[t] = 0.f;
    int jb = 0;
    for (int s = 0; s < a.nsp; ++s) {
      const int beg = a.seg_offs[atom * a.nsp + s];
      const int end = a.seg_offs[atom * a.nsp + s + 1];
      const unsigned char* gsp = g16 + (size_t)s * t16 * RB;
      for (int pbase = beg; pbase < end; pbase += 32, ++jb) {
        if (jb % W != warp) continue;
        const int pidx = pbase + lane;
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
        {
          float f[NC + LC + 1], df[NC + LC + 1];
          table_interp<NC, LC, true>(a.table, a.ti, r, f, df);
          float bn[NC], dbn[NC];
          float bmax = 0.f;
#pragma unroll
          for (int n = 0; n < NC; ++n) {
            const bool on = live && (EXACT || n < nmax);
            bn[n] = on ? f[n] : 0.f;
            dbn[n] = on ? df[n] : 0.f;
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
          __syncwarp();  // previous batch done with bv / ild
          write_split_row<NC, KP, true>(bv, lane, bn);
          write_split_row<NC, KP, true>(bv + 32 * RB, lane, dbn);
#pragma unroll
          for (int l = 0; l < LP; ++l) {
            ild[l * 32 + lane] = f[NC + l];
            ild[(LP + l) * 32 + lane] = df[NC + l];
          }
          __syncwarp();
        }

        // u / u' for tau rows [16 c, 16 c + 16) of all 32 pairs -> ubuf.  Entry (tau pair
        // p = tau / 2, pair j) sits at ubuf[p % 8][j ^ (tau & 6)]: the XOR spreads the 8
        // lanes of each 128-bit store phase over distinct banks.
        auto refill = [&](int chunk) {
          __syncwarp();
          const int mi = lane >> 3, rr = lane & 7;
          uint32_t bf[2][KS][2];
#pragma unroll
          for (int ks = 0; ks < KS; ++ks) {
            const int trow = chunk * 16 + (mi >> 1) * 8 + rr;
            ldsm_x4(smem_u32(gsp + RL::off(trow, 2 * ks + (mi & 1))), bf[0][ks][0], bf[0][ks][1],
                    bf[1][ks][0], bf[1][ks][1]);
          }
          const int g = lane >> 2, t = lane & 3;
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            uint32_t af[2][KS][4];
#pragma unroll
            for (int wh = 0; wh < 2; ++wh)
#pragma unroll
              for (int ks = 0; ks < KS; ++ks) {
                const int prow = mt * 16 + (mi & 1) * 8 + rr;
                ldsm_x4(smem_u32(bv + wh * 32 * RB + RL::off(prow, 2 * ks + (mi >> 1))),
                        af[wh][ks][0], af[wh][ks][1], af[wh][ks][2], af[wh][ks][3]);
              }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
              float du[4] = {0.f, 0.f, 0.f, 0.f}, dp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
              for (int ks = 0; ks < KS; ++ks) {
                mma_f16(du, af[0][ks], bf[nt][ks][0], bf[nt][ks][1]);
                mma_f16(dp, af[1][ks], bf[nt][ks][0], bf[nt][ks][1]);
              }
              float4* ub = ubuf + (nt * 4 + t) * 32 + ((mt * 16 + g) ^ (2 * t));
              ub[0] = make_float4(du[0], dp[0], du[1], dp[1]);
              ub[8] = make_float4(du[2], dp[2], du[3], dp[3]);
            }
          }
          __syncwarp();
        };

        const float* il_l = ild + lane;
        float srad = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
        if constexpr (EXACT) {
          const float4* const ubx[4] = {ubuf + lane, ubuf + (lane ^ 2), ubuf + (lane ^ 4), ubuf + (lane ^ 6)};
          adj_sweep_unrolled<LC>(a.yc, ux, uy, uz, il_l, ubx, refill, srad, hx, hy, hz);
        } else {
        int tau = 0;
        // m = 0 column: N~_l^0 and its z-derivative d[l][0] N~_l^1
        {
          float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f, R = 0.f, Z = 0.f;
          const float2* ub2 = reinterpret_cast<const float2*>(ubuf);
#pragma unroll 1
          for (int l = 0; l <= lmax; ++l, ++tau) {
            const float4 cp = cf.p[l][0], cq = cf.q[l][0];
            const float pl = fmaf(cp.x * uz, a1, fmaf(-cp.y, a2, cq.x));
            a2 = a1;
            a1 = pl;
            const float ql = fmaf(cp.z * uz, b1, fmaf(-cp.w, b2, cq.y));
            b2 = b1;
            b1 = ql;
            const float dz = cq.z * ql;
            const float il = il_l[l * 32], dil = il_l[(LP + l) * 32];
            if ((tau & 15) == 0) refill(tau >> 4);
            const float2 u = ub2[(((tau >> 1) & 7) * 32 + (lane ^ (tau & 6))) * 2 + (tau & 1)];
            R = fmaf(fmaf(u.y, il, u.x * dil), pl, R);
            Z = fmaf(u.x * il, dz, Z);
          }
          srad = R;
          hz = Z;
          tau = tE;
        }
        // m >= 1: cos-type (l, m) at tau, sin-type (l, -m) at tau + 1
        {
          float cm = 1.f, sm = 0.f;
#pragma unroll 1
          for (int m = 1; m <= lmax; ++m) {
            const float cmm1 = cm, smm1 = sm;
            cm = ux * cmm1 - uy * smm1;
            sm = ux * smm1 + uy * cmm1;
            float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
            float Rc = 0.f, Rs = 0.f, Xc = 0.f, Xs = 0.f, Zc = 0.f, Zs = 0.f;
#pragma unroll 1
            for (int l = m; l <= lmax; ++l, tau += 2) {
              const float4 cp = cf.p[l][m], cq = cf.q[l][m];
              const float pl = fmaf(cp.x * uz, a1, fmaf(-cp.y, a2, cq.x));
              a2 = a1;
              a1 = pl;
              const float ql = fmaf(cp.z * uz, b1, fmaf(-cp.w, b2, cq.y));
              b2 = b1;
              b1 = ql;
              const float dz = cq.z * ql;
              const float il = il_l[l * 32], dil = il_l[(LP + l) * 32];
              if ((tau & 15) == 0) refill(tau >> 4);
              const float4 u = ubuf[((tau >> 1) & 7) * 32 + (lane ^ (tau & 6))];
              const float wc = u.x * il, ws = u.z * il;
              Rc = fmaf(fmaf(u.y, il, u.x * dil), pl, Rc);
              Rs = fmaf(fmaf(u.w, il, u.z * dil), pl, Rs);
              Xc = fmaf(wc, pl, Xc);
              Xs = fmaf(ws, pl, Xs);
              Zc = fmaf(wc, dz, Zc);
              Zs = fmaf(ws, dz, Zs);
            }
            // Y_c = P cos, Y_s = P sin with grad_xy from d(rho^m cos/sin m phi)
            const float fm = (float)m;
            srad = fmaf(Rc, cm, fmaf(Rs, sm, srad));
            hx = fmaf(fm, fmaf(Xc, cmm1, Xs * smm1), hx);
            hy = fmaf(fm, fmaf(Xs, cmm1, -Xc * smm1), hy);
            hz = fmaf(Zc, cm, fmaf(Zs, sm, hz));
          }
        }
        }  // rolled sweep
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
  }
}

template <int NC, int LC, int W, bool EXACT>
cudaError_t launch_mma(const AdjArgs<float>& a, cudaStream_t st) {
  const MmaLayout lay = make_layout<NC, LC, W>(a.nsp, EXACT ? NC : a.nmax, EXACT ? LC : a.lmax, a.dim);
  if (lay.total > 220 * 1024) return cudaErrorInvalidConfiguration;
  auto kern = pair_adj_mma_kernel<NC, LC, W, EXACT>;
  cudaError_t e = sg_set_smem<pair_adj_mma_kernel<NC, LC, W, EXACT>>(lay.total);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, lay.total);
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)sms * per_sm;
  if (grid > a.n_atoms) grid = a.n_atoms;
  kern<<<(unsigned)grid, W * 32, lay.total, st>>>(a, lay);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

// Warps per block = 32-pair batches of a typical atom (the warps of a block share one atom).
template <int NC, int LC, bool EXACT>
cudaError_t launch_mma_w(const AdjArgs<float>& a, cudaStream_t st) {
  if (a.warps == 2) return launch_mma<NC, LC, 2, EXACT>(a, st);
  if (a.warps == 3) return launch_mma<NC, LC, 3, EXACT>(a, st);
  if (a.warps == 4) return launch_mma<NC, LC, 4, EXACT>(a, st);
  const int batches = sg_adj_batches_per_atom(a.n_pairs, a.n_atoms, a.nsp);
  if (batches <= 2) return launch_mma<NC, LC, 2, EXACT>(a, st);
  if (batches == 3) return launch_mma<NC, LC, 3, EXACT>(a, st);
  return launch_mma<NC, LC, 4, EXACT>(a, st);
}

template <int NC, int LC>
cudaError_t launch_mma_v(const AdjArgs<float>& a, cudaStream_t st) {
  if (a.nmax == NC && a.lmax == LC) return launch_mma_w<NC, LC, true>(a, st);
  return launch_mma_w<NC, LC, false>(a, st);
}

}  // namespace

int sg_adj_batches_per_atom(long long n_pairs, int n_atoms, int nsp) {
  if (n_atoms <= 0 || nsp <= 0) return 1;
  const double per_seg = (double)n_pairs / ((double)n_atoms * nsp);
  return nsp * (int)std::ceil(per_seg / 32.0);
}

cudaError_t sg_pair_adjoint_mma(const AdjArgs<float>& a, int cls, cudaStream_t st) {
  if (a.n_atoms == 0) return cudaSuccess;
  if (a.warps == SG_ADJ_TCGEN05) {
    if (sg_pair_adjoint_tc_supported(a, cls)) return sg_pair_adjoint_tc(a, cls, st);
    AdjArgs<float> b = a;  // other basis sizes: the mma.sync kernel with four warps
    b.warps = 4;
    return sg_pair_adjoint_mma(b, cls, st);
  }
  switch (cls) {
    case 0: return launch_mma_v<6, 6>(a, st);
    case 1: return launch_mma_v<8, 8>(a, st);
    case 2: return launch_mma_v<10, 10>(a, st);
    default: return launch_mma_v<12, 12>(a, st);
  }
}
