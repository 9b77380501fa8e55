// Power spectrum and normalised descriptor (Eq. 09 and Sec. I), one warp per atom.
//   p[c1][c2][l] = sum_{m=-l..l} c[c1][lm] c[c2][lm]   (real Y_lm: same value as Eq. 09)
//   packed entry (c1 <= c2, l) = p times sqrt(2) when c1 != c2;  q = p / |p|.
#include <algorithm>

#include "internal.h"

// Optional GAP operand of the mixed path (op.a16 set): from q in shared memory, u = (q - qbar)
// / |q - qbar| in FP16 ([hi] or [hi | hi | lo] by op.terms), |q - qbar| and qbar.(q - qbar),
// in the operation order of prep_atoms_kernel (gap_tc.cu).
template <typename T>
__device__ __forceinline__ void gap_operand(const GapOperand& op, int atom, const T* qs, int D, int lane) {
  float s2 = 0.f, dq = 0.f;
  for (int k = lane; k < D; k += 32) {
    const float t = (float)qs[k] - op.qbar[k];
    s2 = fmaf(t, t, s2);
    dq = fmaf(t, op.qbar[k], dq);
  }
  s2 = warp_sum(s2);
  dq = warp_sum(dq);
  const float nn = sqrtf(s2);
  const float iv = nn > 0.f ? 1.f / nn : 0.f;
  __half* row = op.a16 + (size_t)atom * op.terms * op.dp;
  for (int k = lane; k < op.dp; k += 32) {
    const float uk = k < D ? ((float)qs[k] - op.qbar[k]) * iv : 0.f;
    const __half hi = __float2half_rn(uk);
    row[k] = hi;
    if (op.terms == 3) {
      row[op.dp + k] = hi;
      row[2 * op.dp + k] = __float2half_rn(uk - __half2float(hi));
    }
  }
  if (lane == 0) {
    op.nrm[atom] = nn;
    op.uq[atom] = dq;
  }
}

// LC: the basis class's bound on l_max (the (l, m) loops unrolled to it, l_max <= LC at run time)
template <typename T, int LC>
__global__ void powspec_kernel(const T* __restrict__ c, int n_atoms, int nch, int lmax,
                               int per_warp, T* q, T* pnorm, GapOperand op) {
  // one warp per atom: c staged in shared memory, each lane owns whole channel pairs
  // (c1 <= c2) and all their l, the unnormalised p stays in shared memory until |p| is known
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* cs = reinterpret_cast<T*>(smem_raw) + (size_t)warp * per_warp;
  const int L = (lmax + 1) * (lmax + 1);
  const int lp1 = lmax + 1;
  const int npair = nch * (nch + 1) / 2;
  const int D = npair * lp1;
  T* ps = cs + nch * L;
  const T SQRT2 = (T)1.4142135623730951;
  const int wpb = blockDim.x >> 5;
  for (int atom = blockIdx.x * wpb + warp; atom < n_atoms; atom += gridDim.x * wpb) {
    const T* ci = c + (size_t)atom * nch * L;
    __syncwarp();
    for (int k = lane; k < nch * L; k += 32) cs[k] = __ldg(ci + k);
    __syncwarp();
    T ss = 0;
    for (int pc = lane; pc < npair; pc += 32) {
      int c1 = 0, rem = pc;
      while (rem >= nch - c1) {
        rem -= nch - c1;
        ++c1;
      }
      const int c2 = c1 + rem;
      const T* a = cs + c1 * L;
      const T* b = cs + c2 * L;
      const T f = c1 != c2 ? SQRT2 : T(1);
      T* out = ps + pc * lp1;
#pragma unroll
      for (int l = 0; l <= LC; ++l) {
        if (l <= lmax) {
          // two partial sums: the m terms of one l are independent products
          T v0 = 0, v1 = 0;
#pragma unroll
          for (int m = 0; m <= 2 * l; ++m) {
            if (m & 1) v1 = fma(a[l * l + m], b[l * l + m], v1);
            else v0 = fma(a[l * l + m], b[l * l + m], v0);
          }
          const T v = (v0 + v1) * f;
          out[l] = v;
          ss += v * v;
        }
      }
    }
    ss = warp_sum(ss);
    const T norm = sqrt(ss);
    if (lane == 0) pnorm[atom] = norm;
    const T inv = T(1) / norm;
    __syncwarp();
    T* qi = q + (size_t)atom * D;
    for (int k = lane; k < D; k += 32) {
      const T v = ps[k] * inv;
      qi[k] = v;
      if (op.a16) ps[k] = v;  // q, kept for the GAP operand
    }
    if (op.a16) {
      __syncwarp();
      gap_operand<T>(op, atom, ps, D, lane);
    }
  }
}

template <typename T, int LC>
static cudaError_t launch_powspec(const T* c, int n_atoms, int nch, int lmax, T* q, T* pnorm, cudaStream_t st,
                                  const GapOperand& op) {
  if (n_atoms == 0) return cudaSuccess;
  const int L = (lmax + 1) * (lmax + 1);
  const int D = nch * (nch + 1) / 2 * (lmax + 1);
  const int per_warp = (nch * L + D + 3) / 4 * 4;
  const size_t warp_bytes = (size_t)per_warp * sizeof(T);
  int wpb = (int)std::min<size_t>(4, (200 * 1024) / warp_bytes);
  if (wpb < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = warp_bytes * wpb;
  auto kern = powspec_kernel<T, LC>;
  cudaError_t e = sg_set_smem<powspec_kernel<T, LC>>(smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)sms * per_sm;
  const long long need = (n_atoms + wpb - 1) / wpb;
  if (grid > need) grid = need;
  kern<<<(unsigned)grid, wpb * 32, smem, st>>>(c, n_atoms, nch, lmax, per_warp, q, pnorm, op);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

template <typename T>
cudaError_t sg_power_spectrum(const T* c, int n_atoms, int nch, int lmax, int lc, T* q, T* pnorm, cudaStream_t st,
                              const GapOperand& op) {
  if (lmax > lc) return cudaErrorInvalidValue;
  switch (lc) {
    case 6: return launch_powspec<T, 6>(c, n_atoms, nch, lmax, q, pnorm, st, op);
    case 8: return launch_powspec<T, 8>(c, n_atoms, nch, lmax, q, pnorm, st, op);
    case 10: return launch_powspec<T, 10>(c, n_atoms, nch, lmax, q, pnorm, st, op);
    case 12: return launch_powspec<T, 12>(c, n_atoms, nch, lmax, q, pnorm, st, op);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t sg_power_spectrum<float>(const float*, int, int, int, int, float*, float*, cudaStream_t,
                                              const GapOperand&);
template cudaError_t sg_power_spectrum<double>(const double*, int, int, int, int, double*, double*, cudaStream_t,
                                               const GapOperand&);
