// Forces, per-atom energies and per-structure sums.
//   F_k = -dE/dx_k = sum_{pairs p of centre k} (dE/dr_p - dE/dr_rev(p))
// where rev(p) is the reversed pair (j, k, -S): every pair that has k as its neighbour is
// the reverse of a pair centred on k, so the gather is deterministic (no atomics).
// E_struct and the virial are summed per structure in FP64.
#include "internal.h"

// Accumulator of the per-atom sums: FP64 for the FP64 path; for FP32 inputs a double-float
// pair (hi, lo) updated with the exact two-sum, which keeps close to FP64 accuracy without
// FP64 instructions (those are slow on this GPU).
template <typename T> struct SumAcc {
  double v = 0;
  __device__ void add(T x) { v += (double)x; }
  __device__ void warp_reduce() { v = warp_sum(v); }
  __device__ double value() const { return v; }
};
template <> struct SumAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ void add2(float xh, float xl) {
    const float s = hi + xh;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (xh - bp);
    hi = s;
    lo += e + xl;
  }
  __device__ void add(float x) { add2(x, 0.f); }
  __device__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
      const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
      add2(oh, ol);
    }
  }
  __device__ double value() const { return (double)hi + (double)lo; }
};

template <typename T>
__global__ void atom_finish_kernel(int n, int nsp, const int* __restrict__ seg_offs,
                                   const int* __restrict__ pair_idx,
                                   const int* __restrict__ rev, const Vec4<T>* __restrict__ dedr,
                                   const T* __restrict__ eps_part, int n_tiles, T* e_atom,
                                   double* forces, double fsign) {
  // one warp per atom: lanes stride over the atom's pairs (coalesced), then warp sums
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  if (eps_part && e_atom) {
    SumAcc<T> e;
    for (int t = lane; t < n_tiles; t += 32) e.add(eps_part[(size_t)i * n_tiles + t]);
    e.warp_reduce();
    if (lane == 0) e_atom[i] = (T)e.value();
  }
  if (forces) {
    SumAcc<T> f0, f1, f2;
    const int beg = seg_offs[i * nsp], end = seg_offs[(i + 1) * nsp];
    for (int k = beg + lane; k < end; k += 32) {
      const int p = pair_idx ? pair_idx[k] : k;
      const Vec4<T> a = dedr[p], b = dedr[rev[p]];
      f0.add(a.x);
      f0.add(-b.x);
      f1.add(a.y);
      f1.add(-b.y);
      f2.add(a.z);
      f2.add(-b.z);
    }
    f0.warp_reduce();
    f1.warp_reduce();
    f2.warp_reduce();
    if (lane == 0) {
      forces[3 * i] = fsign * f0.value();
      forces[3 * i + 1] = fsign * f1.value();
      forces[3 * i + 2] = fsign * f2.value();
    }
  }
}

#define FINISH_CHUNK 2048

// Partial sums of (e_atom, virial) over chunk blockIdx.y of structure blockIdx.x; a fixed
// order of sums in both levels keeps the result deterministic.
template <typename T>
__global__ void struct_partial_kernel(const int64_t* __restrict__ offs, const T* __restrict__ e_atom,
                                      const T* __restrict__ vir_atom, double* part, int chunks) {
  const int s = blockIdx.x, c = blockIdx.y;
  const int64_t a = offs[s] + (int64_t)c * FINISH_CHUNK;
  const int64_t b = min(offs[s + 1], a + FINISH_CHUNK);
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
    part[((size_t)s * chunks + c) * 10 + threadIdx.x] = v;
  }
}

// one warp per structure: lanes take chunks c = lane, lane + 32, ..., then a fixed-order
// shuffle tree (deterministic)
__global__ void struct_total_kernel(int n_struct, int chunks, const double* __restrict__ part,
                                    double* e_struct, double* virial) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= n_struct) return;
  double acc[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) acc[t] = 0;
  for (int c = lane; c < chunks; c += 32)
#pragma unroll
    for (int t = 0; t < 10; ++t) acc[t] += part[((size_t)s * chunks + c) * 10 + t];
#pragma unroll
  for (int t = 0; t < 10; ++t) acc[t] = warp_sum(acc[t]);
  if (lane == 0) {
    if (e_struct) e_struct[s] = acc[0];
    if (virial)
      for (int t = 0; t < 9; ++t) virial[(size_t)s * 9 + t] = acc[1 + t];
  }
}

int sg_finish_chunks(int max_struct_atoms) {
  return max_struct_atoms <= 0 ? 1 : (max_struct_atoms + FINISH_CHUNK - 1) / FINISH_CHUNK;
}

template <typename T>
cudaError_t sg_finish(int n_atoms, int n_struct, int nsp, const int64_t* atom_offs_dev,
                      const int* seg_offs, const int* pair_idx, const int* rev, const Vec4<T>* dedr,
                      const T* eps_part, int n_tiles, const T* vir_atom, T* e_atom,
                      double* e_struct, double* forces, double* virial, bool sign_force,
                      int chunks, double* part, cudaStream_t st) {
  if (n_atoms > 0 && ((eps_part && e_atom) || forces)) {
    atom_finish_kernel<T><<<(n_atoms * 32 + 255) / 256, 256, 0, st>>>(
        n_atoms, nsp, seg_offs, pair_idx, rev, dedr, eps_part, n_tiles, e_atom, forces,
        sign_force ? 1.0 : -1.0);
    ++sg_kernel_launches;
  }
  if (n_struct > 0 && (e_struct || virial)) {
    struct_partial_kernel<T><<<dim3(n_struct, chunks), 256, 0, st>>>(
        atom_offs_dev, e_struct ? e_atom : nullptr, virial ? vir_atom : nullptr, part, chunks);
    struct_total_kernel<<<(n_struct * 32 + 127) / 128, 128, 0, st>>>(n_struct, chunks, part, e_struct, virial);
    sg_kernel_launches += 2;
  }
  return cudaGetLastError();
}

template cudaError_t sg_finish<float>(int, int, int, const int64_t*, const int*, const int*, const int*,
                                      const Vec4<float>*, const float*, int, const float*, float*,
                                      double*, double*, double*, bool, int, double*, cudaStream_t);
template cudaError_t sg_finish<double>(int, int, int, const int64_t*, const int*, const int*, const int*,
                                       const Vec4<double>*, const double*, int, const double*,
                                       double*, double*, double*, double*, bool, int, double*, cudaStream_t);

// ---------------------------------------------------------------- velocity Verlet
// Units: positions A, velocities A/fs, forces eV/A, masses amu, time fs.
// 1 eV/(A amu) = 0.009648533212 A/fs^2.
#define SG_EV_PER_AMU_A2_FS2 0.009648533212

// kick: v += (dt/2) F/m;  with drift: then x += dt v.  Positions are not wrapped: the
// neighbour-list build maps them into their cells itself, and unwrapped positions keep a
// Verlet-skin list valid when atoms cross a cell face.
__global__ void verlet_kernel(int n, double* __restrict__ pos, double* __restrict__ vel,
                              const double* __restrict__ forces, const double* __restrict__ inv_mass,
                              double dt, int drift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double kick = 0.5 * dt * SG_EV_PER_AMU_A2_FS2 * inv_mass[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double v = vel[3 * i + c] + kick * forces[3 * i + c];
    vel[3 * i + c] = v;
    if (drift) pos[3 * i + c] += dt * v;
  }
}

cudaError_t sg_verlet(int n, double* pos, double* vel, const double* forces, const double* inv_mass,
                      double dt, bool drift, cudaStream_t st) {
  if (n > 0) {
    verlet_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, pos, vel, forces, inv_mass, dt, drift ? 1 : 0);
    ++sg_kernel_launches;
  }
  return cudaGetLastError();
}
