// GAP local energies for callers that cannot allocate device memory.
//
// The regular path keeps its scratch (per-tile partial energy sums) in a workspace that
// the handle grows with cudaMalloc.  This entry point runs the same GAP energy kernel
// but takes its scratch from a fixed array in the library's own device memory, so the
// call itself allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/soapgap.h"
#include "internal.h"

// Scratch: per-tile partial sums, n_atoms x ceil(m / 64) floats, at most 4 Mi floats
// (16 MiB).  Every GPU that loads the library holds this array until the process exits.
#define SG_NOALLOC_SCRATCH_FLOATS (4u << 20)
// The energy kernel covers 64 atoms per block row, and a grid has at most 65535 rows.
#define SG_NOALLOC_MAX_ATOMS (65535 * 64)
static __device__ __align__(256) float g_noalloc_scratch[SG_NOALLOC_SCRATCH_FLOATS];

// Host code cannot use g_noalloc_scratch directly (on the host that name is a stand-in,
// not a device address).  Its device address is looked up once per device and context:
// a device reset destroys the context and the module with it, and the array may come
// back at another address in the next context.  Contexts are told apart by the driver's
// context ID, which is never reused within a process.
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

static std::mutex g_noalloc_mu;
static float* g_noalloc_ptr[256];
static unsigned long long g_noalloc_ctx[256];
static ctx_get_current_fn g_ctx_get_current;
static ctx_get_id_fn g_ctx_get_id;

static bool resolve_driver_calls() {
  if (g_ctx_get_current && g_ctx_get_id) return true;
  void* a = nullptr;
  void* b = nullptr;
  cudaDriverEntryPointQueryResult qa, qb;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 4000, cudaEnableDefault, &qa) !=
          cudaSuccess ||
      qa != cudaDriverEntryPointSuccess || !a)
    return false;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) !=
          cudaSuccess ||
      qb != cudaDriverEntryPointSuccess || !b)
    return false;
  g_ctx_get_current = reinterpret_cast<ctx_get_current_fn>(a);
  g_ctx_get_id = reinterpret_cast<ctx_get_id_fn>(b);
  return true;
}

static int noalloc_scratch(float** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SOAPGAP_E_CUDA;
  // makes the device's primary context current on this thread (no allocation)
  if (cudaSetDevice(dev) != cudaSuccess) return SOAPGAP_E_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!resolve_driver_calls()) return SOAPGAP_E_CUDA;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS)
    return SOAPGAP_E_CUDA;
  if (!g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SOAPGAP_E_CUDA;
    g_noalloc_ptr[dev] = static_cast<float*>(p);
    g_noalloc_ctx[dev] = id;
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
  if ((unsigned long long)n * (unsigned long long)tiles > SG_NOALLOC_SCRATCH_FLOATS ||
      n > SG_NOALLOC_MAX_ATOMS)
    return SOAPGAP_E_CAPACITY;
  float* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != SOAPGAP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // an error left by earlier, unrelated work is not this call's: clear it before launching
  (void)cudaGetLastError();
  // every partial sum is written before it is read: nothing in the scratch needs zeroing
  if (sg_gap_forward_simt<float>(q, q_sparse, alpha, n, m, d, zeta, scratch, tiles, nullptr, st) !=
      cudaSuccess)
    return SOAPGAP_E_CUDA;
  noalloc_rowsum<<<(n + 255) / 256, 256, 0, st>>>(scratch, n, tiles, e_atom);
  if (cudaPeekAtLastError() != cudaSuccess) return SOAPGAP_E_CUDA;
  ++sg_kernel_launches;
  return SOAPGAP_OK;
}
