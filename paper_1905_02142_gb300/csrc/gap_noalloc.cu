// GAP local energies for callers that cannot allocate device memory.
//
// The regular path keeps its scratch (per-tile partial energy sums) in a workspace that
// the handle grows with cudaMalloc.  This entry point runs the same GAP energy kernel
// but takes its scratch from a fixed array in the library's own device memory, so the
// call itself allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/soapgap.h"
#include "internal.h"

// Scratch: per-tile partial sums, n_atoms x ceil(m / 64) floats, at most 4 Mi floats
// (16 MiB).  Every GPU that loads the library holds this array until the process exits.
#define SG_NOALLOC_SCRATCH_FLOATS (4u << 20)
static __device__ __align__(256) float g_noalloc_scratch[SG_NOALLOC_SCRATCH_FLOATS];

// Host code cannot use g_noalloc_scratch directly (on the host that name is a stand-in,
// not a device address); its device address is looked up once per device.
static std::mutex g_noalloc_mu;
static float* g_noalloc_ptr[256];

static int noalloc_scratch(float** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SOAPGAP_E_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SOAPGAP_E_CUDA;
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return SOAPGAP_OK;
}

__global__ void noalloc_rowsum(const float* __restrict__ part, int n, int tiles, float* e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int t = 0; t < tiles; ++t) s += (double)part[(size_t)i * tiles + t];
  e[i] = (float)s;
}

extern "C" int soapgap_gap_energy_noalloc(const float* q, const float* q_sparse, const float* alpha,
                                          int32_t n, int32_t m, int32_t d, double zeta,
                                          float* e_atom, void* stream) {
  if (n < 0 || m < 1 || d < 1 || !(zeta > 0)) return SOAPGAP_E_INVALID_ARG;
  if (n == 0) return SOAPGAP_OK;
  if (!q || !q_sparse || !alpha || !e_atom) return SOAPGAP_E_INVALID_ARG;
  const int tiles = sg_gap_tiles(m);
  if ((unsigned long long)n * (unsigned long long)tiles > SG_NOALLOC_SCRATCH_FLOATS)
    return SOAPGAP_E_CAPACITY;
  float* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != SOAPGAP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // every partial sum is written before it is read: nothing in the scratch needs zeroing
  if (sg_gap_forward_simt<float>(q, q_sparse, alpha, n, m, d, zeta, scratch, tiles, nullptr, st) !=
      cudaSuccess)
    return SOAPGAP_E_CUDA;
  noalloc_rowsum<<<(n + 255) / 256, 256, 0, st>>>(scratch, n, tiles, e_atom);
  ++sg_kernel_launches;
  return cudaGetLastError() == cudaSuccess ? SOAPGAP_OK : SOAPGAP_E_CUDA;
}
