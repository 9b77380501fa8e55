// GAP model on CUDA cores (FP64 path, and the FP32 reference variant of the mixed path).
//   S = Q Qs^T,  eps_i = sum_s alpha_s S_is^zeta   (Sec. IV.A, SOAP kernel of Sec. I)
//   kp_is = zeta alpha_s S_is^(zeta-1),  g = kp Qs = dE/dq   (adjoint of the above)
// Classic 64x64 register-tiled GEMM, 256 threads, 4x4 outputs per thread.
#include "internal.h"

#define GB_M 64
#define GB_N 64
#define GB_K 16

int sg_gap_tiles(int m) { return (m + GB_N - 1) / GB_N; }

template <typename T> __device__ __forceinline__ T kpow(T s, int izeta, T zeta) {
  if (izeta > 0) {
    T o = s;
    for (int k = 1; k < izeta; ++k) o *= s;
    return o;
  }
  return pow(s > T(0) ? s : T(0), zeta);
}

// MODE 0: C = A B^T (A [M,K], B [N,K]) with the GAP forward epilogue
// MODE 1: C = A B   (A [M,K], B [K,N]) plain store
template <typename T, int MODE>
__global__ void __launch_bounds__(256)
gemm_kernel(const T* __restrict__ A, const T* __restrict__ B, int M, int N, int K,
            const T* __restrict__ alpha, int izeta, T zeta, T* eps_part, int n_tiles, T* out,
            int ldo) {
  __shared__ T As[GB_K][GB_M + 4];
  __shared__ T Bs[GB_K][GB_N + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.y * GB_M, col0 = blockIdx.x * GB_N;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int k0 = 0; k0 < K; k0 += GB_K) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t;            // 0..1023
      const int r = e >> 4, kk = e & 15;      // A tile: 64 rows x 16 k
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? A[(size_t)gr * K + gk] : T(0);
      if (MODE == 0) {
        const int gc = col0 + r;
        Bs[kk][r] = (gc < N && gk < K) ? B[(size_t)gc * K + gk] : T(0);
      } else {
        const int kb = e >> 6, c = e & 63;    // B tile: 16 k x 64 cols
        const int gkb = k0 + kb, gc = col0 + c;
        Bs[kb][c] = (gkb < K && gc < N) ? B[(size_t)gkb * N + gc] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (MODE == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gr = row0 + ty + 16 * i;
      T part = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gc = col0 + tx + 16 * j;
        if (gr < M && gc < N) {
          const T s = acc[i][j], al = alpha[gc];
          const T sz1 = (izeta == 1) ? T(1) : kpow(s, izeta > 0 ? izeta - 1 : 0, zeta - T(1));
          const T sz = (izeta > 0) ? sz1 * s : kpow(s, 0, zeta);
          part += al * sz;
          if (out) out[(size_t)gr * ldo + gc] = zeta * al * sz1;
        }
      }
      // reduce over the 16 threads of this row (tx = lane & 15)
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (tx == 0 && gr < M) eps_part[(size_t)gr * n_tiles + blockIdx.x] = part;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gr = row0 + ty + 16 * i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gc = col0 + tx + 16 * j;
        if (gr < M && gc < N) out[(size_t)gr * ldo + gc] = acc[i][j];
      }
    }
  }
}

template <typename T>
cudaError_t sg_gap_forward_simt(const T* q, const T* qs, const T* alpha, int n, int m, int d,
                                double zeta, T* eps_part, int n_tiles, T* kp, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int iz = (zeta >= 1.0 && zeta == (double)(int)zeta) ? (int)zeta : 0;
  dim3 grid(sg_gap_tiles(m), (n + GB_M - 1) / GB_M);
  gemm_kernel<T, 0><<<grid, 256, 0, st>>>(q, qs, n, m, d, alpha, iz, (T)zeta, eps_part, n_tiles,
                                          kp, m);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

template <typename T>
cudaError_t sg_gap_backward_simt(const T* kp, const T* qs, int n, int m, int d, T* g,
                                 cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  dim3 grid((d + GB_N - 1) / GB_N, (n + GB_M - 1) / GB_M);
  gemm_kernel<T, 1><<<grid, 256, 0, st>>>(kp, qs, n, d, m, nullptr, 0, T(0), nullptr, 0, g, d);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

template cudaError_t sg_gap_forward_simt<float>(const float*, const float*, const float*, int, int,
                                                int, double, float*, int, float*, cudaStream_t);
template cudaError_t sg_gap_forward_simt<double>(const double*, const double*, const double*, int,
                                                 int, int, double, double*, int, double*, cudaStream_t);
template cudaError_t sg_gap_backward_simt<float>(const float*, const float*, int, int, int, float*,
                                                 cudaStream_t);
template cudaError_t sg_gap_backward_simt<double>(const double*, const double*, int, int, int,
                                                  double*, cudaStream_t);
