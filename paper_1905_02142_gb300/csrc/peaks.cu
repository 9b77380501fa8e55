// Arithmetic peaks of the device, measured: the denominators of the roofline of the pair
// kernels (FP32 FMA) and of the FP64 path (FP64 FMA).
//
// Every thread runs eight independent chains of fused multiply-adds, x <- x a + b, with
// 0 < a < 1 so the values settle at b / (1 - a) and stay normal.  Eight chains per thread
// and eight blocks of 256 threads per SM keep every FMA pipe fed whatever its latency.
// Work per launch: 2 flop x 8 chains x 16 (unrolled) x iters x threads.
#include <cuda_runtime.h>

#include "../../include/soapgap.h"
#include "internal.h"

namespace {

__device__ float g_peak_sink_f;
__device__ double g_peak_sink_d;

template <typename T>
__global__ void __launch_bounds__(256) alu_peak_kernel(int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-6, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = fma(x0, a, b);
      x1 = fma(x1, a, b);
      x2 = fma(x2, a, b);
      x3 = fma(x3, a, b);
      x4 = fma(x4, a, b);
      x5 = fma(x5, a, b);
      x6 = fma(x6, a, b);
      x7 = fma(x7, a, b);
    }
  }
  const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == (T)-1) {  // never true (every chain stays positive): keeps the chains live
    if constexpr (sizeof(T) == 4)
      g_peak_sink_f = (float)s;
    else
      g_peak_sink_d = (double)s;
  }
}

template <typename T>
int measure(int iters, T a, T b, double* tflops, int32_t* sm_count, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return SOAPGAP_E_CUDA;
  const int blocks = sms * 8, threads = 256;
  const double flop = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return SOAPGAP_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SOAPGAP_E_CUDA;
  }
  float best = -1.f;
  int rc = SOAPGAP_OK;
  for (int rep = 0; rep < 4 && rc == SOAPGAP_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, st);
    alu_peak_kernel<T><<<blocks, threads, 0, st>>>(iters, a, b);
    ++sg_kernel_launches;
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = SOAPGAP_E_CUDA;
      break;
    }
    if (rep > 0 && (best < 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SOAPGAP_OK) return rc;
  *tflops = flop / (best * 1e-3) / 1e12;
  if (sm_count) *sm_count = sms;
  return SOAPGAP_OK;
}

}  // namespace

extern "C" int soapgap_measure_alu_peak(int32_t kind, double* tflops, int32_t* sm_count, void* stream) {
  if (!tflops) return SOAPGAP_E_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (kind == SOAPGAP_PEAK_FP32_FMA) return measure<float>(4096, 0.9999999f, 1e-7f, tflops, sm_count, st);
  if (kind == SOAPGAP_PEAK_FP64_FMA) return measure<double>(96, 0.9999999, 1e-7, tflops, sm_count, st);
  return SOAPGAP_E_INVALID_ARG;
}
