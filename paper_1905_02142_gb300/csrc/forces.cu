// Forces, per-atom energies and per-structure sums.
//   F_k = -dE/dx_k = sum_{pairs p of centre k} (dE/dr_p - dE/dr_rev(p))
// where rev(p) is the reversed pair (j, k, -S): every pair that has k as its neighbour is
// the reverse of a pair centred on k, so the gather is deterministic (no atomics).
// E_struct and the virial are summed per structure in FP64.
#include "internal.h"

template <typename T>
__global__ void atom_finish_kernel(int n, int nsp, const int* __restrict__ seg_offs,
                                   const int* __restrict__ rev, const Vec4<T>* __restrict__ dedr,
                                   const T* __restrict__ eps_part, int n_tiles, T* e_atom,
                                   double* forces, double fsign) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (eps_part && e_atom) {
    double e = 0;
    for (int t = 0; t < n_tiles; ++t) e += (double)eps_part[(size_t)i * n_tiles + t];
    e_atom[i] = (T)e;
  }
  if (forces) {
    double f[3] = {0, 0, 0};
    const int beg = seg_offs[i * nsp], end = seg_offs[(i + 1) * nsp];
    for (int p = beg; p < end; ++p) {
      const Vec4<T> a = dedr[p], b = dedr[rev[p]];
      f[0] += (double)a.x - (double)b.x;
      f[1] += (double)a.y - (double)b.y;
      f[2] += (double)a.z - (double)b.z;
    }
    forces[3 * i] = fsign * f[0];
    forces[3 * i + 1] = fsign * f[1];
    forces[3 * i + 2] = fsign * f[2];
  }
}

template <typename T>
__global__ void struct_finish_kernel(const int64_t* __restrict__ offs, const T* __restrict__ e_atom,
                                     const T* __restrict__ vir_atom, double* e_struct,
                                     double* virial) {
  const int s = blockIdx.x;
  const int64_t a = offs[s], b = offs[s + 1];
  double acc[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) acc[t] = 0;
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
    if (e_atom) acc[0] += (double)e_atom[i];
    if (vir_atom)
#pragma unroll
      for (int t = 0; t < 9; ++t) acc[1 + t] += (double)vir_atom[i * 9 + t];
  }
  __shared__ double red[10][8];
#pragma unroll
  for (int t = 0; t < 10; ++t) {
    double v = warp_sum(acc[t]);
    if ((threadIdx.x & 31) == 0) red[t][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    if (threadIdx.x == 0) {
      if (e_struct) e_struct[s] = v;
    } else if (virial) {
      virial[(size_t)s * 9 + threadIdx.x - 1] = v;
    }
  }
}

template <typename T>
cudaError_t sg_finish(int n_atoms, int n_struct, int nsp, const int64_t* atom_offs_dev,
                      const int* seg_offs, const int* rev, const Vec4<T>* dedr,
                      const T* eps_part, int n_tiles, const T* vir_atom, T* e_atom,
                      double* e_struct, double* forces, double* virial, bool sign_force,
                      cudaStream_t st) {
  if (n_atoms > 0 && ((eps_part && e_atom) || forces)) {
    atom_finish_kernel<T><<<(n_atoms + 127) / 128, 128, 0, st>>>(
        n_atoms, nsp, seg_offs, rev, dedr, eps_part, n_tiles, e_atom, forces,
        sign_force ? 1.0 : -1.0);
    ++sg_kernel_launches;
  }
  if (n_struct > 0 && (e_struct || virial)) {
    struct_finish_kernel<T><<<n_struct, 256, 0, st>>>(atom_offs_dev, e_struct ? e_atom : nullptr,
                                                      virial ? vir_atom : nullptr, e_struct, virial);
    ++sg_kernel_launches;
  }
  return cudaGetLastError();
}

template cudaError_t sg_finish<float>(int, int, int, const int64_t*, const int*, const int*,
                                      const Vec4<float>*, const float*, int, const float*, float*,
                                      double*, double*, double*, bool, cudaStream_t);
template cudaError_t sg_finish<double>(int, int, int, const int64_t*, const int*, const int*,
                                       const Vec4<double>*, const double*, int, const double*,
                                       double*, double*, double*, double*, bool, cudaStream_t);
