// Power spectrum and normalised descriptor (Eq. 09 and Sec. I), one block per atom.
//   p[c1][c2][l] = sum_{m=-l..l} c[c1][lm] c[c2][lm]   (real Y_lm: same value as Eq. 09)
//   packed entry (c1 <= c2, l) = p times sqrt(2) when c1 != c2;  q = p / |p|.
#include "internal.h"

template <typename T>
__global__ void powspec_kernel(const T* __restrict__ c, int nch, int lmax, T* q, T* pnorm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* cs = reinterpret_cast<T*>(smem_raw);
  __shared__ T red[32];
  const int atom = blockIdx.x;
  const int L = (lmax + 1) * (lmax + 1);
  const int lp1 = lmax + 1;
  const int npair = nch * (nch + 1) / 2;
  const int D = npair * lp1;
  const T* ci = c + (size_t)atom * nch * L;
  for (int k = threadIdx.x; k < nch * L; k += blockDim.x) cs[k] = ci[k];
  __syncthreads();
  T* qi = q + (size_t)atom * D;
  T ss = 0;
  const T SQRT2 = (T)1.4142135623730951;
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    const int pc = k / lp1, l = k - pc * lp1;
    int c1 = 0, rem = pc;
    while (rem >= nch - c1) { rem -= nch - c1; ++c1; }
    const int c2 = c1 + rem;
    const T* a = cs + c1 * L + l * l;
    const T* b = cs + c2 * L + l * l;
    T v = 0;
    for (int m = 0; m < 2 * l + 1; ++m) v = fma(a[m], b[m], v);
    if (c1 != c2) v *= SQRT2;
    qi[k] = v;
    ss += v * v;
  }
  ss = warp_sum(ss);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    T t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
    t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  const T norm = sqrt(red[0]);
  if (threadIdx.x == 0) pnorm[atom] = norm;
  const T inv = T(1) / norm;
  for (int k = threadIdx.x; k < D; k += blockDim.x) qi[k] *= inv;
}

template <typename T>
cudaError_t sg_power_spectrum(const T* c, int n_atoms, int nch, int lmax, T* q, T* pnorm,
                              cudaStream_t st) {
  if (n_atoms == 0) return cudaSuccess;
  const int L = (lmax + 1) * (lmax + 1);
  const size_t smem = (size_t)nch * L * sizeof(T);
  auto kern = powspec_kernel<T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<n_atoms, 128, smem, st>>>(c, nch, lmax, q, pnorm);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

template cudaError_t sg_power_spectrum<float>(const float*, int, int, int, float*, float*, cudaStream_t);
template cudaError_t sg_power_spectrum<double>(const double*, int, int, int, double*, double*, cudaStream_t);
