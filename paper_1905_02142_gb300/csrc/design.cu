// Sparse-GAP fitting matrices (Sec. IV.A: the weights alpha_s are fitted to the energies and
// forces of training environments, with the sparse environments as basis; SOAP kernel of
// Sec. I):
//   k(i, s)     = (q_i . q_s)^zeta                          kernel rows (K_NM)
//   kt(t, s)    = sum over the atoms i of structure t of k(i, s)      energy rows
//   dk(k, a, s) = d/dx_{k,a} sum over i in the structure of k of k(i, s)   force rows
//
// Force rows by forward differentiation of the descriptors.  With p_i the unnormalised
// power spectrum (q_i = p_i / |p_i|) and J_ij = dp_i/dr_ij (D x 3) for r_ij = x_j + S h - x_i,
//   dk(i, s)/dr_ij = w_is (q_s - S_is q_i) . J_ij,    w_is = zeta S_is^(zeta-1) / |p_i|,
// and x_j moves r_ij by +1, x_i by -1, so for a target atom k
//   dk(k, ., s) = sum over pairs (j -> k) of w_js (q_s - S_js q_j) . J_jk
//               + w_ks (q_s - S_ks q_k) . J_k,self,        J_k,self = -sum_j J_kj.
// The columns (3 per pair, 3 self columns per atom) are stored by TARGET: atom k owns the
// column range [3 (o_k + k), 3 (o_(k+1) + k + 1)), o_k its first pair in the list; the pair
// (j -> k) fills the slot of its reverse (k -> j), the self columns come last.  A GEMM of
// the sparse rows against all columns then applies the owner's weights and sums each
// target's columns in its epilogue (gap_tc.cu for the mixed path, dgemm_nt_kernel here).
//
// Mixed path: since (q_s - S q_o) . J = q_s . J' with J' = J - q_o (q_o . J) (the part of J
// orthogonal to q_o), the columns are projected in FP32 before they are rounded, and stored
// as FP16 [2^e J' | hi, lo of 2^e qbar . J'] with one power of two per column triple.  The
// sparse operand is [kd (q_s - qbar) | kd | kd], so the tensor cores return kd 2^e q_s . J'
// with the large common part qbar . J' carried exactly; the epilogue only scales by
// w_os 2^-e / kd.  FP64 path: unprojected columns and (w, w S) weights on q_s . J and q_o . J.
//
// Per pair, with c_(ch, lm) += b_n(r) A_lm(r_vec), A_lm = 4 pi ilexp_l Y_lm (Sec. II), for
// the channels ch = (species(j), n) of the pair's block:
//   X[c][l] = sum_m A_lm c_(c, lm),     Z[c][l] = sum_m grad A_lm c_(c, lm)
//   J[(c1, c2, l)] = f ( 1[c1 in block] (b'_n1 rhat X[c2][l] + b_n1 Z[c2][l])
//                      + 1[c2 in block] (b'_n2 rhat X[c1][l] + b_n2 Z[c1][l]) )
// with f = sqrt(2) for c1 != c2 (derivative of the packed power spectrum, Eq. 09), and
// grad A_lm = 4 pi (ilexp_l' Y_lm rhat + ilexp_l (I - rhat rhat^T) grad P_lm / r).
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.h"
#include "soapmath.cuh"
#include "table.cuh"

namespace {

__host__ __device__ constexpr size_t al32(size_t b) { return (b + 31) / 32 * 32; }

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

constexpr int JB = 16;  // pairs per batch of the Jacobian kernel's radial phase

// floats per warp region of the Jacobian kernel (multiple of 4 elements: Vec4 alignment)
template <int NC, int LC>
int jac_per_warp(int nsp, int nmax, int lmax, int dim) {
  constexpr int NP = (NC + 3) / 4 * 4, LP = (LC + 1 + 3) / 4 * 4;
  const int L = (lmax + 1) * (lmax + 1), nch = nsp * nmax, lp1 = lmax + 1;
  const int dpad = (dim + 7) / 8 * 8;  // row stride of the [3][D] arrays (16-byte aligned rows)
  const int jt = std::max(4 * L, 3 * dpad);
  const int n = 4 * nch * lp1 + 4 * JB + (jt + 3) / 4 * 4 + (nch * L + 3) / 4 * 4 + dpad + 3 * dpad +
                JB * (2 * NP + 2 * LP) + 2 * JB;
  return (n + 3) / 4 * 4;
}

// One warp per owner atom i: its pairs one after the other, the warp's lanes sharing the
// work of each (radial terms: lane 0; angular terms: one lane per m; X/Z: lanes over (c, l);
// J: lanes over the packed entries).  Columns are written as FP16 scaled by a power of two
// per column (TABLE, mixed path; max |entry| in [2^14, 2^15)) or FP64 unscaled.
template <typename T, int NC, int LC, bool TABLE>
__global__ void __launch_bounds__(SG_WARPS * 32)
design_jacobian_kernel(const JacArgs<T> a, int per_warp) {
  constexpr int NP = (NC + 3) / 4 * 4, LP = (LC + 1 + 3) / 4 * 4;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nsp = a.nsp, nmax = a.nmax, lmax = a.lmax, D = a.dim;
  const int L = (lmax + 1) * (lmax + 1), nch = nsp * nmax, lp1 = lmax + 1;
  YlmShared<T>& ys = *reinterpret_cast<YlmShared<T>*>(smem_raw);
  size_t off = al32(sizeof(YlmShared<T>));
  int* ddec = reinterpret_cast<int*>(smem_raw + off);  // [D] c1 | c2 << 8 | l << 16
  off += al32(sizeof(int) * D);
  int* edec = reinterpret_cast<int*>(smem_raw + off);  // [nch * lp1] c | l << 8, by decreasing l
  off += al32(sizeof(int) * nch * lp1);
  float* qbar_s = reinterpret_cast<float*>(smem_raw + off);
  off += al32(sizeof(float) * (TABLE ? D : 1));
  T* wbase = reinterpret_cast<T*>(smem_raw + off) + (size_t)warp * per_warp;
  constexpr int RW = 2 * NP + 2 * LP;                // radial record of one pair
  const int Dp = (D + 7) / 8 * 8;  // row stride of the [3][D] arrays (16-byte aligned rows)
  const int jt = (max(4 * L, 3 * Dp) + 3) / 4 * 4;
  Vec4<T>* XZ = reinterpret_cast<Vec4<T>*>(wbase);  // [nch][lp1]  X, Z
  Vec4<T>* geo = XZ + nch * lp1;                     // [JB]  rhat, 1/r (< 0: masked pair)
  T* Jt = reinterpret_cast<T*>(geo + JB);            // [3][Dp] J of the current pair, and before
  Vec4<T>* Aw = reinterpret_cast<Vec4<T>*>(Jt);      //   it [L] A_lm, grad A_lm (used up by X, Z)
  T* cs = Jt + jt;                                   // [nch][L]  c of the owner
  T* qi = cs + (nch * L + 3) / 4 * 4;                // [D]     q of the owner
  T* Jacc = qi + Dp;                                 // [3][Dp] -sum of J (self columns)
  T* rad = Jacc + 3 * Dp;                            // [JB][RW] b_n, b_n', A_l, A_l' per pair
  int* pinfo = reinterpret_cast<int*>(rad + JB * RW);  // [JB][2] first column, neighbour
  const T SQRT2 = (T)1.4142135623730951;

  load_ylm_shared(ys, a.yc);
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    const int pc = d / lp1, l = d - pc * lp1;
    int c1 = 0, rem = pc;
    while (rem >= nch - c1) {
      rem -= nch - c1;
      ++c1;
    }
    ddec[d] = c1 | ((c1 + rem) << 8) | (l << 16);
  }
  // X/Z work items by decreasing l: the lanes of one round then sum over similar m ranges
  for (int e = threadIdx.x; e < nch * lp1; e += blockDim.x) edec[e] = (e % nch) | ((lmax - e / nch) << 8);
  if (TABLE)
    for (int d = threadIdx.x; d < D; d += blockDim.x) qbar_s[d] = a.qbar[d];
  __syncthreads();

  T qmx = 0, qbq = 0;  // per owner atom: max |q_o| and qbar . q_o (set in the atom loop)
  // per-lane partials over the lane's entries of src[3][D]: max |J|, q_owner.J, qbar.J
  auto partials = [&](const T* src, T* mx, T* tq, T* tb) {
#pragma unroll
    for (int c = 0; c < 3; ++c) { mx[c] = T(0); tb[c] = T(0); tq[c] = T(0); }
    for (int d = lane; d < D; d += 32) {
      const T qv = qi[d];
      const T qb = TABLE ? (T)qbar_s[d] : T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T v = src[c * Dp + d];
        mx[c] = max(mx[c], abs(v));
        tq[c] = fma(qv, v, tq[c]);
        tb[c] = fma(qb, v, tb[c]);
      }
    }
  };
  // write the three columns of one pair (or self slot) from src[3][D], given the partials
  auto emit3 = [&](const T* src, long long col0, int owner, int target, T* mx, T* tq, T* tb) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mx[c] = warp_max(mx[c]);
      tq[c] = warp_sum(tq[c]);
      tb[c] = warp_sum(tb[c]);
    }
    T inv_scale[3] = {T(1), T(1), T(1)};
    if constexpr (TABLE) {
      // Projected columns J' = J - q_o (q_o . J) (the force row then needs q_s . J' only,
      // since (q_s - S q_o) . J = q_s . J'), followed by hi and lo of qbar . J' (the sparse
      // operand carries two unit columns there).  One power-of-two scale per triple, from
      // a bound on |J'| = |J - q_o t| <= max |J| + max |q_o| |t| and on |qbar . J'|.
      float sc = 1.f, tbp[3];
      {
        float big = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          tbp[c] = (float)(tb[c] - qbq * tq[c]);
          big = fmaxf(big, fmaxf((float)(mx[c] + qmx * abs(tq[c])), fabsf(tbp[c])));
        }
        const int e = big > 0.f ? 14 - ilogbf(big) : 0;
        sc = ldexpf(1.f, e);
        inv_scale[0] = inv_scale[1] = inv_scale[2] = (T)ldexpf(1.f, -e);
      }
      // 8 halves per lane and step over the pieces inside [0, D): rows of src and q_o read as
      // 16-byte vectors, one 16-byte store.  The piece holding D and the two carried terms is
      // written by lane c of the three; the padding after it stays zero from allocation.
      const int full8 = D / 8;
      __half* rows = reinterpret_cast<__half*>(a.J) + (size_t)col0 * a.ld;
      for (int q = lane; q < 3 * full8; q += 32) {
        const int c = (q >= full8) + (q >= 2 * full8);
        const int k8 = q - c * full8;
        const float tcs = (float)(c == 0 ? tq[0] : (c == 1 ? tq[1] : tq[2])) * sc;
        const T* sp = src + c * Dp + 8 * k8;
        const T* qp = qi + 8 * k8;
        const float4 s0 = *reinterpret_cast<const float4*>(sp), s1 = *reinterpret_cast<const float4*>(sp + 4);
        const float4 q0 = *reinterpret_cast<const float4*>(qp), q1 = *reinterpret_cast<const float4*>(qp + 4);
        __align__(16) __half2 h4[4];
        h4[0] = __floats2half2_rn(fmaf(-q0.x, tcs, s0.x * sc), fmaf(-q0.y, tcs, s0.y * sc));
        h4[1] = __floats2half2_rn(fmaf(-q0.z, tcs, s0.z * sc), fmaf(-q0.w, tcs, s0.w * sc));
        h4[2] = __floats2half2_rn(fmaf(-q1.x, tcs, s1.x * sc), fmaf(-q1.y, tcs, s1.y * sc));
        h4[3] = __floats2half2_rn(fmaf(-q1.z, tcs, s1.z * sc), fmaf(-q1.w, tcs, s1.w * sc));
        *reinterpret_cast<uint4*>(rows + (size_t)c * a.ld + 8 * k8) = *reinterpret_cast<const uint4*>(h4);
      }
      if (lane < 3) {
        // entries 8 full8 .. D + 1 of column c (at most 9: D mod 8 + 2), within the row since
        // ld >= D + 2
        const int c = lane;
        const float tcs = (float)(c == 0 ? tq[0] : (c == 1 ? tq[1] : tq[2])) * sc;
        const float xb = (c == 0 ? tbp[0] : (c == 1 ? tbp[1] : tbp[2])) * sc;
        const __half xh = __float2half_rn(xb);
        __half* row = rows + (size_t)c * a.ld;
        for (int d = 8 * full8; d < D; ++d)
          row[d] = __float2half_rn(fmaf(-(float)qi[d], tcs, (float)src[c * Dp + d] * sc));
        row[D] = xh;
        row[D + 1] = __float2half_rn(xb - __half2float(xh));
      }
    } else {
      double* rows = reinterpret_cast<double*>(a.J) + (size_t)col0 * a.ld;
      for (int q = lane; q < 3 * a.ld; q += 32) {
        const int c = (q >= a.ld) + (q >= 2 * a.ld);
        const int d = q - c * a.ld;
        rows[q] = d < D ? (double)src[c * Dp + d] : 0.0;
      }
    }
    if (lane < 3) {
      const int c = lane;
      const T tbc = c == 0 ? tb[0] : (c == 1 ? tb[1] : tb[2]);
      const T tqc = c == 0 ? tq[0] : (c == 1 ? tq[1] : tq[2]);
      const T isc = c == 0 ? inv_scale[0] : (c == 1 ? inv_scale[1] : inv_scale[2]);
      a.col_at[col0 + c] = make_int2(owner, target);
      a.col_v[col0 + c] = Vec4<T>{tbc, tqc, isc, T(0)};
    }
  };

  const int wpb = blockDim.x >> 5;
  for (int atom = blockIdx.x * wpb + warp; atom < a.n_atoms; atom += gridDim.x * wpb) {
    __syncwarp();
    const T* ci = a.c + (size_t)atom * nch * L;
    for (int k = lane; k < nch * L; k += 32) cs[k] = ci[k];
    const T* qrow = a.q + (size_t)atom * D;
    qmx = 0;
    qbq = 0;
    for (int d = lane; d < D; d += 32) {
      const T qv = qrow[d];
      qi[d] = qv;
      qmx = max(qmx, abs(qv));
      if (TABLE) qbq = fma((T)qbar_s[d], qv, qbq);
      Jacc[d] = Jacc[Dp + d] = Jacc[2 * Dp + d] = T(0);
    }
    qmx = warp_max(qmx);
    qbq = warp_sum(qbq);
    __syncwarp();
    for (int sj = 0; sj < nsp; ++sj) {
      const int beg = a.seg_offs[atom * nsp + sj], end = a.seg_offs[atom * nsp + sj + 1];
      const int blk0 = sj * nmax;
      for (int base = beg; base < end; base += JB) {
        // ---- per batch of JB pairs, one lane each: geometry, columns, radial terms
        {
          const int p = base + lane;
          if (lane < JB && p < end) {
            const Vec4<T> v = a.pair_r[p];
            const int j = a.pair_j[p];
            pinfo[2 * lane] = 3 * (a.rev[p] + j);
            pinfo[2 * lane + 1] = j;
            // |r| < 0 marks a pair beyond r_cut in a list built with a skin: zero columns
            const bool live = v.w >= T(0);
            const T r = live ? v.w : T(1), inv = T(1) / r;
            geo[lane] = Vec4<T>{live ? v.x * inv : T(0), live ? v.y * inv : T(0), live ? v.z * inv : T(1),
                                live ? inv : T(-1)};
            T* rr = rad + lane * RW;
            if constexpr (TABLE) {
              float f[NC + LC + 1], df[NC + LC + 1];
              table_interp<NC, LC, true>(a.table, a.ti, (float)r, f, df);
#pragma unroll
              for (int n = 0; n < NP; ++n) {
                rr[n] = n < NC ? (T)f[n] : T(0);
                rr[NP + n] = n < NC ? (T)df[n] : T(0);
              }
#pragma unroll
              for (int l = 0; l < LP; ++l) {
                rr[2 * NP + l] = l <= LC ? (T)f[NC + l] : T(0);
                rr[2 * NP + LP + l] = l <= LC ? (T)df[NC + l] : T(0);
              }
            } else {
              using Dd = Dual<double>;
              Dd rd((double)r, 1.0);
              Dd ba[NC];
              radial_alpha<Dd, NC>(rd, a.p, ba);
#pragma unroll
              for (int n = 0; n < NC; ++n) {
                double bv = 0.0, bd = 0.0;
#pragma unroll
                for (int al = 0; al < NC; ++al) {
                  bv = fma((double)a.bc.W[n][al], ba[al].v, bv);
                  bd = fma((double)a.bc.W[n][al], ba[al].d, bd);
                }
                rr[n] = (T)(n < nmax ? bv : 0.0);
                rr[NP + n] = (T)(n < nmax ? bd : 0.0);
              }
              Dd spp = a.p.s0p + a.p.ap * rd;
              Dd ild[LC + 1];
              ilexp_all<Dd, LC>(rd * rd / (spp * spp), ild);
#pragma unroll
              for (int l = 0; l <= LC; ++l) {
                const double wl = (l <= lmax) ? 12.566370614359172 * (a.p.eq08 ? (2.0 * l + 1.0) : 1.0) : 0.0;
                rr[2 * NP + l] = (T)(wl * ild[l].v);
                rr[2 * NP + LP + l] = (T)(wl * ild[l].d);
              }
            }
          }
        }
        __syncwarp();
        const int cnt = min(JB, end - base);
        for (int k = 0; k < cnt; ++k) {
          const Vec4<T> g = geo[k];
          const T* bs = rad + k * RW;
          const T* dbs = bs + NP;
          const T* ils = bs + 2 * NP;
          const T* dils = ils + LP;
          const T ux = g.x, uy = g.y, uz = g.z, inv = g.w;
          T mx[3], tq[3], tb[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) { mx[c] = T(0); tq[c] = T(0); tb[c] = T(0); }
          if (inv > T(0)) {
            // ---- angular terms: lanes m and 16 + m run column m of the harmonic recursion,
            // the first writing the +m (and m = 0) terms, the second the -m terms
            const int m = lane & 15;
            const bool neg = lane >= 16;
            if (m <= lmax && !(neg && m == 0)) {
              T cm = 1, sm = 0, cmm1 = 0, smm1 = 0;
              for (int t = 1; t <= m; ++t) {
                const T c2 = ux * cm - uy * sm, s2 = ux * sm + uy * cm;
                cmm1 = cm;
                smm1 = sm;
                cm = c2;
                sm = s2;
              }
              auto put = [&](int lm, T il, T dil, T y, T gx, T gy, T gz) {
                const T gd = gx * ux + gy * uy + gz * uz;
                const T rr = dil * y, tt = il * inv;
                Aw[lm] = Vec4<T>{il * y, fma(rr, ux, tt * (gx - gd * ux)), fma(rr, uy, tt * (gy - gd * uy)),
                                 fma(rr, uz, tt * (gz - gd * uz))};
              };
              T a2 = 0, a1 = ys.seed[m], b2 = 0, b1 = ys.seed[m + 1];
              const T fm = (T)m;
              for (int l = m; l <= lmax; ++l) {
                T pl, ql = T(0);
                if (l == m) {
                  pl = a1;
                } else {
                  pl = (l == m + 1) ? ys.s1[m] * uz * a1 : ys.a[l][m] * uz * a1 - ys.b[l][m] * a2;
                  a2 = a1;
                  a1 = pl;
                  if (l == m + 1) {
                    ql = b1;
                  } else {
                    ql = (l == m + 2) ? ys.s1[m + 1] * uz * b1 : ys.a[l][m + 1] * uz * b1 - ys.b[l][m + 1] * b2;
                    b2 = b1;
                    b1 = ql;
                  }
                }
                const T dz = ys.d[l][m] * ql;
                const T il = ils[l], dil = dils[l];
                const int l0 = l * l + l;
                if (m == 0) {
                  put(l0, il, dil, pl, T(0), T(0), dz);
                } else {
                  const T pm = fm * pl;
                  if (!neg) put(l0 + m, il, dil, pl * cm, pm * cmm1, -pm * smm1, dz * cm);
                  else put(l0 - m, il, dil, pl * sm, pm * smm1, pm * cmm1, dz * sm);
                }
              }
            }
            __syncwarp();
            // ---- X and Z for every channel and l
            for (int e = lane; e < nch * lp1; e += 32) {
              const int ec = edec[e];
              const int c2 = ec & 0xff, l = ec >> 8;
              const T* crow = cs + c2 * L;
              T x = 0, zx = 0, zy = 0, zz = 0;
              for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) {
                const Vec4<T> w4 = Aw[lm];
                const T cv = crow[lm];
                x = fma(w4.x, cv, x);
                zx = fma(w4.y, cv, zx);
                zy = fma(w4.z, cv, zy);
                zz = fma(w4.w, cv, zz);
              }
              XZ[c2 * lp1 + l] = Vec4<T>{x, zx, zy, zz};
            }
            __syncwarp();
            // ---- J over the packed entries (c1 <= c2, l), with the lane's partials
            for (int d = lane; d < D; d += 32) {
              const int cc = ddec[d];
              const int c1 = cc & 0xff, c2 = (cc >> 8) & 0xff, l = cc >> 16;
              const int n1 = c1 - blk0, n2 = c2 - blk0;
              T j0 = 0, j1 = 0, j2 = 0;
              if ((unsigned)n1 < (unsigned)nmax) {
                const Vec4<T> z = XZ[c2 * lp1 + l];
                const T br = dbs[n1] * z.x, b0 = bs[n1];
                j0 = fma(br, ux, b0 * z.y);
                j1 = fma(br, uy, b0 * z.z);
                j2 = fma(br, uz, b0 * z.w);
              }
              if ((unsigned)n2 < (unsigned)nmax) {
                const Vec4<T> z = XZ[c1 * lp1 + l];
                const T br = dbs[n2] * z.x, b0 = bs[n2];
                j0 += fma(br, ux, b0 * z.y);
                j1 += fma(br, uy, b0 * z.z);
                j2 += fma(br, uz, b0 * z.w);
              }
              const T f = c1 == c2 ? T(1) : SQRT2;
              const T jv[3] = {j0 * f, j1 * f, j2 * f};
              const T qv = qi[d];
              const T qb = TABLE ? (T)qbar_s[d] : T(0);
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                Jt[c * Dp + d] = jv[c];
                Jacc[c * Dp + d] -= jv[c];
                mx[c] = max(mx[c], abs(jv[c]));
                tq[c] = fma(qv, jv[c], tq[c]);
                tb[c] = fma(qb, jv[c], tb[c]);
              }
            }
          } else {
            for (int d = lane; d < 3 * Dp; d += 32) Jt[d] = T(0);
          }
          __syncwarp();
          emit3(Jt, (long long)pinfo[2 * k], atom, pinfo[2 * k + 1], mx, tq, tb);
          __syncwarp();
        }
      }
    }
    const int ie = a.seg_offs[(atom + 1) * nsp];
    {
      T mx[3], tq[3], tb[3];
      partials(Jacc, mx, tq, tb);
      emit3(Jacc, 3LL * ((long long)ie + atom), atom, atom, mx, tq, tb);
    }
  }
}

template <typename T, int NC, int LC, bool TABLE>
cudaError_t launch_jacobian(const JacArgs<T>& a, cudaStream_t st) {
  const int per_warp = jac_per_warp<NC, LC>(a.nsp, a.nmax, a.lmax, a.dim);
  const int nch = a.nsp * a.nmax;
  const size_t head = al32(sizeof(YlmShared<T>)) + al32(sizeof(int) * (size_t)a.dim) +
                      al32(sizeof(int) * (size_t)nch * (a.lmax + 1)) + al32(sizeof(float) * (TABLE ? a.dim : 1));
  // up to SG_WARPS warps per block, fewer when their regions do not fit in 220 KB
  const size_t limit = 220 * 1024, warp_bytes = (size_t)per_warp * sizeof(T);
  if (head + warp_bytes > limit) return cudaErrorInvalidConfiguration;
  const int wpb = (int)std::min<size_t>(SG_WARPS, (limit - head) / warp_bytes);
  const size_t smem = head + (size_t)wpb * warp_bytes;
  auto kern = design_jacobian_kernel<T, NC, LC, TABLE>;
  cudaError_t e = sg_set_smem<design_jacobian_kernel<T, NC, LC, TABLE>>(smem);
  if (e != cudaSuccess) return e;
  // all of the SM's shared memory for this kernel: one more block per SM for common sizes
  static bool carved = false;
  if (!carved) {
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    carved = true;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
  if (per_sm < 1) per_sm = 1;
  long long need = (a.n_atoms + wpb - 1) / wpb;
  long long grid = (long long)sms * per_sm * 4;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, wpb * 32, smem, st>>>(a, per_warp);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 contraction
// C[r][c] = sum_k A[r][k] B[c][k] (row-major FP64), 64 x 64 tiles, 256 threads holding 4 x 4
// outputs each; epi(r, c, C) for every r < m, c < n.
template <class Epi>
__global__ void __launch_bounds__(256)
dgemm_nt_kernel(const double* __restrict__ A, int m, const double* __restrict__ B, long long n, int k, Epi epi) {
  __shared__ double As[16][65], Bs[16][65];
  const int r0 = blockIdx.y * 64;
  const long long c0 = (long long)blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < k; k0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      const int kk = t & 15, rr = t >> 4;
      const bool kin = k0 + kk < k;
      As[kk][rr] = (r0 + rr < m && kin) ? A[(size_t)(r0 + rr) * k + k0 + kk] : 0.0;
      Bs[kk][rr] = (c0 + rr < n && kin) ? B[(size_t)(c0 + rr) * k + k0 + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i;
      const long long c = c0 + tx * 4 + j;
      if (r < m && c < n) epi(r, c, acc[i][j]);
    }
}

__device__ __forceinline__ double pow_zeta(double s, double zeta, int izeta) {
  if (izeta > 0) {
    double o = s;
    for (int t = 1; t < izeta; ++t) o *= s;
    return o;
  }
  return pow(fmax(s, 0.0), zeta);
}

// kernel rows: k(i, s) and the force-row weights (w_is, w_is S_is)
struct EpiRows64 {
  int M, ldw, izeta;
  double zeta;
  const double* pnorm;
  double* k;
  double2* wv;
  __device__ void operator()(int i, long long s, double S) const {
    k[(size_t)i * M + s] = pow_zeta(S, zeta, izeta);
    if (wv) {
      const double w = zeta * (izeta == 1 ? 1.0 : pow_zeta(S, zeta - 1.0, izeta - 1)) / pnorm[i];
      wv[(size_t)i * ldw + s] = make_double2(w, w * S);
    }
  }
};

// force rows: one column's contribution to its target (FP64 atomics)
struct EpiDk64 {
  int M, ldw;
  const int2* col_at;
  const Vec4<double>* col_v;
  const double2* wv;
  double* dk;
  __device__ void operator()(int s, long long col, double C) const {
    const int2 at = col_at[col];
    const double2 w = wv[(size_t)at.x * ldw + s];
    const double val = w.x * C - w.y * col_v[col].y;
    atomicAdd(dk + ((size_t)at.y * 3 + (size_t)(col % 3)) * M + s, val);
  }
};

template <class Epi>
cudaError_t launch_dgemm(const double* A, int m, const double* B, long long n, int k, Epi epi, cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const long long gx = (n + 63) / 64;
  if (gx > 0x7fffffffLL || (m + 63) / 64 > 65535) return cudaErrorInvalidConfiguration;
  dgemm_nt_kernel<Epi><<<dim3((unsigned)gx, (unsigned)((m + 63) / 64)), 256, 0, st>>>(A, m, B, n, k, epi);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

// per-structure sums of kernel rows (atom chunks of 128 per block, FP64 atomics per
// structure segment within a chunk)
template <typename T>
__global__ void struct_rows_kernel(const T* __restrict__ k, int n, int m, const int* __restrict__ atom_struct,
                                   double* out) {
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  const int a0 = blockIdx.x * 128, a1 = min(n, a0 + 128);
  if (s >= m || a0 >= n) return;
  double acc = 0.0;
  int cur = atom_struct[a0];
  for (int i = a0; i < a1; ++i) {
    const int t = atom_struct[i];
    if (t != cur) {
      atomicAdd(out + (size_t)cur * m + s, acc);
      acc = 0.0;
      cur = t;
    }
    acc += (double)k[(size_t)i * m + s];
  }
  atomicAdd(out + (size_t)cur * m + s, acc);
}

}  // namespace

template <typename T>
cudaError_t sg_design_jacobian(const JacArgs<T>& a, int cls, bool table, cudaStream_t st) {
  if (a.n_atoms == 0) return cudaSuccess;
  if (table) {
    if constexpr (sizeof(T) == 4) {
      switch (cls) {
        case 0: return launch_jacobian<T, 6, 6, true>(a, st);
        case 1: return launch_jacobian<T, 8, 8, true>(a, st);
        case 2: return launch_jacobian<T, 10, 10, true>(a, st);
        default: return launch_jacobian<T, 12, 12, true>(a, st);
      }
    }
    return cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 8) {
    switch (cls) {
      case 0: return launch_jacobian<T, 6, 6, false>(a, st);
      case 1: return launch_jacobian<T, 8, 8, false>(a, st);
      case 2: return launch_jacobian<T, 10, 10, false>(a, st);
      default: return launch_jacobian<T, 12, 12, false>(a, st);
    }
  }
  return cudaErrorInvalidValue;
}

template cudaError_t sg_design_jacobian<float>(const JacArgs<float>&, int, bool, cudaStream_t);
template cudaError_t sg_design_jacobian<double>(const JacArgs<double>&, int, bool, cudaStream_t);

cudaError_t sg_kernel_rows_f64(const double* q, int n, const double* qs, int m, int d, double zeta,
                               const double* pnorm, double* k, double2* wv, int ldw, cudaStream_t st) {
  EpiRows64 e{};
  e.M = m;
  e.ldw = ldw;
  e.izeta = (zeta >= 1.0 && zeta == (double)(int)zeta) ? (int)zeta : 0;
  e.zeta = zeta;
  e.pnorm = pnorm;
  e.k = k;
  e.wv = wv;
  return launch_dgemm(q, n, qs, m, d, e, st);
}

cudaError_t sg_design_grad_f64(const double* qs, int m, int d, const double* J, long long ncols,
                               const int2* col_at, const Vec4<double>* col_v, const double2* wv, int ldw,
                               double* dk, cudaStream_t st) {
  EpiDk64 e{m, ldw, col_at, col_v, wv, dk};
  return launch_dgemm(qs, m, J, ncols, d, e, st);
}

template <typename T>
cudaError_t sg_struct_rows(const T* k, int n, int m, const int* atom_struct, double* out, cudaStream_t st) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  const int gy = (m + 255) / 256;
  if (gy > 65535) return cudaErrorInvalidConfiguration;
  struct_rows_kernel<T><<<dim3((unsigned)((n + 127) / 128), (unsigned)gy), 256, 0, st>>>(k, n, m, atom_struct, out);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

template cudaError_t sg_struct_rows<float>(const float*, int, int, const int*, double*, cudaStream_t);
template cudaError_t sg_struct_rows<double>(const double*, int, int, const int*, double*, cudaStream_t);
