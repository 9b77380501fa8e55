// Adjoint pair kernel of the FP64 path: dE/dq -> dE/dp -> dE/dc -> dE/dr_ij for every
// pair, recomputing the pair's radial and angular terms instead of storing dc/dr.  (The
// mixed-precision path runs the same mathematics in pair_adj_mma.cu.)
//
// Per atom (one warp):
//   h      = dE/dp = (g - q (q.g)) / |p|                          (q = p/|p|, Sec. I)
//   G_l    = M_l c_l with M_l[c][c] = 2 h_(c,c,l), M_l[c][c'] = sqrt(2) h_(min,max,l)
//            (derivative of the packed power spectrum, Eq. 09)   -> dE/dc[ch][lm]
//   recursion path: G_alpha = W^T G_n (c_n = W c_alpha, Sec. III.A)
// Per pair (one lane), with c_nlm += b_n(r) a_lm(r_vec), a_lm = 4 pi ilexp_l(z(r)) Y_lm(r_hat):
//   u_lm  = sum_n G[n][lm] b_n,   u'_lm = sum_n G[n][lm] b_n'(r)
//   dE/dr_vec = r_hat sum_lm (u'_lm il_l + u_lm il_l') Y_lm
//             + (1/r)(I - r_hat r_hat^T) sum_lm u_lm il_l grad_u P_lm
// where P_lm is the polynomial extension of Y_lm off the sphere.  The radial derivatives
// come from forward-mode duals through Eq. 04.
#pragma once
#include <algorithm>

#include "internal.h"
#include "soapmath.cuh"

// EXACT: n_max == NC and l_max == LC (no runtime size guards in the channel loops).
template <typename T, int NC, int LC, bool EXACT>
__global__ void __launch_bounds__(SG_WARPS * 32)
pair_adj_kernel(const AdjArgs<T> a, int smem_per_warp) {
  constexpr int NP = (NC + 3) / 4 * 4;
  constexpr int LP = LC + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  YlmShared<T>& ys = *reinterpret_cast<YlmShared<T>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* base_s = reinterpret_cast<T*>(smem_raw + (sizeof(YlmShared<T>) + 15) / 16 * 16) + (size_t)warp * smem_per_warp;
  const int L = (a.lmax + 1) * (a.lmax + 1);
  const int nch = a.nsp * a.nmax;
  const int D = a.dim;
  const int lp1 = a.lmax + 1;
  T* Gs = base_s;                          // [nsp][L][NP]   dE/dc, one row of NP per (s, lm)
  T* scratch = Gs + (size_t)a.nsp * L * NP;
  T* cs = scratch;                         // prologue: [nch][L] coefficients
  T* hs = cs + (size_t)nch * L;            //           [D] dE/dp
  T* il_s = scratch;                       // pair loop: [LP][32] ilexp, then [LP][32] d/dr
  T* dil_s = scratch + LP * 32;
  const T FOUR_PI = (T)12.566370614359172;
  const T SQRT2 = (T)1.4142135623730951;

  load_ylm_shared(ys, a.yc);  // recursion coefficients -> shared memory (once per block)
  __syncthreads();

  for (int atom = blockIdx.x * SG_WARPS + warp; atom < a.n_atoms; atom += gridDim.x * SG_WARPS) {
    // ---- prologue: dE/dc in shared memory
    const T w = (T)a.struct_w[a.atom_struct[atom]];
    const T* qi = a.q + (size_t)atom * D;
    const T* gi = a.g + (size_t)atom * D;
    T dot = 0;
    for (int k = lane; k < D; k += 32) dot += qi[k] * gi[k];
    dot = warp_sum(dot);
    const T inv_norm = T(1) / a.pnorm[atom];
    for (int k = lane; k < D; k += 32) hs[k] = w * (gi[k] - qi[k] * dot) * inv_norm;
    const T* ci = a.c + (size_t)atom * nch * L;
    for (int k = lane; k < nch * L; k += 32) cs[k] = ci[k];
    __syncwarp();
    // G[c1][lm] = sum_c2 M_l[c1][c2] c[c2][lm]; packed pair (c1<=c2) index = rowoff(c1) + c2
    for (int lm = lane; lm < L; lm += 32) {
      const int l = (int)sqrtf((float)lm + 0.5f);
      for (int s = 0; s < a.nsp; ++s) {
        T acc[NC];
#pragma unroll
        for (int n = 0; n < NC; ++n) acc[n] = T(0);
        for (int c2 = 0; c2 < nch; ++c2) {
          const T cv = cs[c2 * L + lm];
          const int roff2 = c2 * nch - c2 * (c2 + 1) / 2;  // pc(c2, c1) = roff2 + c1 for c1 >= c2
#pragma unroll
          for (int n = 0; n < NC; ++n) {
            if (EXACT || n < a.nmax) {
              const int c1 = s * a.nmax + n;
              const int pc = c1 >= c2 ? roff2 + c1 : c1 * nch - c1 * (c1 + 1) / 2 + c2;
              const T hv = hs[pc * lp1 + l];
              acc[n] = fma(c1 == c2 ? T(2) * hv : SQRT2 * hv, cv, acc[n]);
            }
          }
        }
        T* grow = Gs + ((size_t)s * L + lm) * NP;
#pragma unroll
        for (int n = 0; n < NP; ++n) grow[n] = (n < NC && (EXACT || n < a.nmax)) ? acc[n] : T(0);
      }
    }
    __syncwarp();
    {
      // G_alpha = W^T G_n (lane-local per (s, lm) row)
      for (int k = lane; k < a.nsp * L; k += 32) {
        T gn[NC];
#pragma unroll
        for (int n = 0; n < NC; ++n) gn[n] = (n < a.nmax) ? Gs[(size_t)k * NP + n] : T(0);
#pragma unroll
        for (int al = 0; al < NC; ++al) {
          T acc = 0;
#pragma unroll
          for (int n = 0; n < NC; ++n) acc = fma(a.bc.W[n][al], gn[n], acc);
          if (al < a.nmax) Gs[(size_t)k * NP + al] = acc;
        }
      }
      __syncwarp();
    }

    // ---- pairs: one lane per pair; the (l, m) loop runs rolled
    T vir[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) vir[t] = 0;
    for (int s = 0; s < a.nsp; ++s) {
      const int beg = a.seg_offs[atom * a.nsp + s];
      const int end = a.seg_offs[atom * a.nsp + s + 1];
      const T* Gsp = Gs + (size_t)s * L * NP;
      for (int pbase = beg; pbase < end; pbase += 32) {
        const int pidx = pbase + lane;
        const bool valid = pidx < end;
        __syncwarp();
        T bn[NC], dbn[NC];
        T ux = 0, uy = 0, uz = 1, r = 1, inv = 1;
        Vec4<T> v{};
        const int pp = (valid && a.pair_idx) ? a.pair_idx[pidx] : pidx;  // index in the full list
        if (valid) v = a.pair_r[pp];
        // |r| < 0 marks a pair beyond r_cut in a list built with a skin: dE/dr = 0
        const bool live = valid && v.w >= T(0);
        if (live) {
          r = v.w;
          inv = T(1) / r;
          ux = v.x * inv; uy = v.y * inv; uz = v.z * inv;
        }
        {
          using Dd = Dual<double>;
          Dd rd((double)r, 1.0);
          Dd ba[NC];
          radial_alpha<Dd, NC>(rd, a.p, ba);
          Dd spp = a.p.s0p + a.p.ap * rd;
          Dd ild[LC + 1];
          ilexp_all<Dd, LC>(rd * rd / (spp * spp), ild);
#pragma unroll
          for (int n = 0; n < NC; ++n) { bn[n] = (T)ba[n].v; dbn[n] = (T)ba[n].d; }
#pragma unroll
          for (int l = 0; l <= LC; ++l) {
            const T wl = (l <= a.lmax) ? FOUR_PI * (T)(a.p.eq08 ? (2.0 * l + 1.0) : 1.0) : T(0);
            il_s[l * 32 + lane] = wl * (T)ild[l].v;
            dil_s[l * 32 + lane] = wl * (T)ild[l].d;
          }
        }
        T srad = 0, hx = 0, hy = 0, hz = 0;
        // one (l, m) term: u = G.b, u' = G.b'; radial and angular contributions
        auto term = [&](int lm, T il, T dil, T y, T gx, T gy, T gz) {
          const T* grow = Gsp + (size_t)lm * NP;
          T gr[NP];
          if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int n = 0; n < NP; n += 4) {
              const float4 g4 = *reinterpret_cast<const float4*>(grow + n);
              gr[n] = g4.x; gr[n + 1] = g4.y; gr[n + 2] = g4.z; gr[n + 3] = g4.w;
            }
          } else {
#pragma unroll
            for (int n = 0; n < NP; n += 2) {
              const double2 g2 = *reinterpret_cast<const double2*>(grow + n);
              gr[n] = g2.x; gr[n + 1] = g2.y;
            }
          }
          T u0 = 0, u1 = 0, v0 = 0, v1 = 0;
#pragma unroll
          for (int n = 0; n < NC; n += 2) {
            u0 = fma(gr[n], bn[n], u0);
            u1 = fma(gr[n], dbn[n], u1);
            if (n + 1 < NC) {
              v0 = fma(gr[n + 1], bn[n + 1], v0);
              v1 = fma(gr[n + 1], dbn[n + 1], v1);
            }
          }
          u0 += v0;
          u1 += v1;
          srad = fma(fma(u1, il, u0 * dil), y, srad);
          const T wv = u0 * il;
          hx = fma(wv, gx, hx);
          hy = fma(wv, gy, hy);
          hz = fma(wv, gz, hz);
        };
        T cm = 1, sm = 0, cmm1 = 0, smm1 = 0;
        const int lmax = EXACT ? LC : a.lmax;
#pragma unroll 1
        for (int m = 0; m <= lmax; ++m) {
          if (m > 0) {
            const T c2 = ux * cm - uy * sm;
            const T s2 = ux * sm + uy * cm;
            cmm1 = cm; smm1 = sm;
            cm = c2; sm = s2;
          }
          T a2 = 0, a1 = ys.seed[m];          // column m of N~ (recursion in l)
          T b2 = 0, b1 = ys.seed[m + 1];      // column m+1 (zero seed past the end)
          const T fm = (T)m;
#pragma unroll 1
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
            const T il = il_s[l * 32 + lane], dil = dil_s[l * 32 + lane];
            const int l0 = l * l + l;
            if (m == 0) {
              term(l0, il, dil, pl, T(0), T(0), dz);
            } else {
              const T pm = fm * pl;
              term(l0 + m, il, dil, pl * cm, pm * cmm1, -pm * smm1, dz * cm);
              term(l0 - m, il, dil, pl * sm, pm * smm1, pm * cmm1, dz * sm);
            }
          }
        }
        if (valid && !live) a.dedr[pp] = Vec4<T>{T(0), T(0), T(0), T(0)};
        if (live) {
          const T hdot = hx * ux + hy * uy + hz * uz;
          Vec4<T> o;
          o.x = ux * srad + (hx - hdot * ux) * inv;
          o.y = uy * srad + (hy - hdot * uy) * inv;
          o.z = uz * srad + (hz - hdot * uz) * inv;
          o.w = T(0);
          a.dedr[pp] = o;
          const T gvec[3] = {o.x, o.y, o.z}, rvec[3] = {v.x, v.y, v.z};
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) vir[3 * p + q2] -= gvec[p] * rvec[q2];
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const T vt = warp_sum(vir[t]);
      if (lane == 0) a.vir_atom[(size_t)atom * 9 + t] = vt;
    }
    __syncwarp();
  }
}

template <typename T, int NC, int LC, bool EXACT>
static cudaError_t launch_adj_v(const AdjArgs<T>& a, cudaStream_t st) {
  constexpr int NP = (NC + 3) / 4 * 4;
  const int L = (a.lmax + 1) * (a.lmax + 1);
  const int nch = a.nsp * a.nmax;
  const int scratch = std::max(nch * L + a.dim, 2 * (LC + 1) * 32);
  int per_warp = a.nsp * L * NP + scratch;
  per_warp = (per_warp + 3) / 4 * 4;
  const size_t smem = (sizeof(YlmShared<T>) + 15) / 16 * 16 + (size_t)SG_WARPS * per_warp * sizeof(T);
  if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
  auto kern = pair_adj_kernel<T, NC, LC, EXACT>;
  cudaError_t e = sg_set_smem<pair_adj_kernel<T, NC, LC, EXACT>>(smem);
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
  kern<<<(unsigned)grid, SG_WARPS * 32, smem, st>>>(a, per_warp);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

template <typename T, int NC, int LC>
static cudaError_t launch_adj(const AdjArgs<T>& a, cudaStream_t st) {
  if (a.nmax == NC && a.lmax == LC) return launch_adj_v<T, NC, LC, true>(a, st);
  return launch_adj_v<T, NC, LC, false>(a, st);
}

template <typename T>
cudaError_t sg_pair_adjoint(const AdjArgs<T>& a, int cls, bool table, cudaStream_t st) {
  if (a.n_atoms == 0) return cudaSuccess;
  if (table) {
    if constexpr (sizeof(T) == 4) return sg_pair_adjoint_mma(a, cls, st);
    return cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 8) {
    switch (cls) {
      case 0: return launch_adj<T, 6, 6>(a, st);
      case 1: return launch_adj<T, 8, 8>(a, st);
      case 2: return launch_adj<T, 10, 10>(a, st);
      default: return launch_adj<T, 12, 12>(a, st);
    }
  }
  return cudaErrorInvalidValue;
}

