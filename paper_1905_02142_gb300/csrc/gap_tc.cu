// GAP model on the tensor cores (mixed-precision path): tcgen05.mma with FP16 operands
// staged by TMA in 128B-swizzled shared memory and FP32 accumulators in tensor memory.
//
//   eps_i = sum_s alpha_s (q_i . q_s)^zeta      (Sec. IV.A with the SOAP kernel of Sec. I)
//   g_i   = dE/dq_i = sum_s zeta alpha_s (q_i . q_s)^(zeta-1) q_s
//
// The dot products q_i.q_s lie close together (0.86..1.0 on carbon-like boxes) and the
// alpha_s have random signs, so eps_i is a strong cancellation: plain BF16 operands lose
// ~6e-2 of it and plain FP16 ~5e-3.  The products are therefore split as
//   q = qbar + n u,  qbar = mean of the sparse rows, n = |q - qbar|, |u| = 1,
//   q_i.q_s = qbar.qbar + qbar.(q_i - qbar) + qbar.(q_s - qbar) + n_i n_s (u_i . u_s),
// with the rank-one terms in FP32 and only u_i.u_s on the tensor cores, either as one FP16
// product hi*hi (K = D) or as the split hi*hi + hi*lo + lo*hi (one GEMM over K = 3 D:
// A = [hi|hi|lo], B = [hi|lo|hi]; relative error ~1e-7 on eps).  How much one product loses
// depends on the model (a few 1e-6 on carbon-like boxes with thousands of sparse rows, above
// 1e-4 with a dozen): the library measures it per model and picks the number of products.
// The backward product needs less: g_i = r_i qbar + kappa kp'_i U with
// r_i = sum_s zeta alpha_s S^(zeta-1) in FP32, kp'_is = zeta alpha_s n_s S^(zeta-1) / kappa in
// FP16 and U the unit sparse rows in FP16 (single pass).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "tcgen05.cuh"

namespace {

constexpr int BM = 128, BK = 64;

using namespace tc5;

// Columns an epilogue takes per TMEM read: Epi::CHUNK (24 or 32) if declared, else 32.
template <class E, class = void> struct EpiChunk { static constexpr int value = 32; };
template <class E> struct EpiChunk<E, std::void_t<decltype(E::CHUNK)>> { static constexpr int value = E::CHUNK; };
// Epilogues with Epi::STAGED write a 32 x 32 FP16 output box per chunk through shared memory
// and a TMA store (two 2 KB staging buffers per epilogue warp).
template <class E, class = void> struct EpiStaged { static constexpr bool value = false; };
template <class E> struct EpiStaged<E, std::void_t<decltype(E::STAGED)>> { static constexpr bool value = E::STAGED; };

// ------------------------------------------------------------------ epilogues
struct EpiStore {  // C = A B^T (diagnostic)
  int rows, cols;
  float* c;
  __device__ void begin(int) {}
  __device__ void apply(int row, int col0, const uint32_t* v) {
    if (row >= rows) return;
    for (int j = 0; j < 32; ++j)
      if (col0 + j < cols) c[(size_t)row * cols + col0 + j] = __uint_as_float(v[j]);
  }
  __device__ void end(int, int) {}
};

// s^(Z-1) for a compile-time integer Z >= 1
template <int Z>
__device__ __forceinline__ float pow_zm1(float s) {
  float o = 1.f;
#pragma unroll
  for (int k = 1; k < Z; ++k) o *= s;
  return o;
}

struct EpiGapFwd {
  static constexpr bool STAGED = true;  // kp through shared memory and TMA stores
  int rows, ld_kp, n_tiles, izeta;
  float zeta;
  const float *u, *nrm;              // [N]
  const float4* col;                 // [Mp] (qbar.qbar + qbar.(q_s-qbar), n_s, alpha_s, f_s)
  float *eps_part, *r_part;          // [N][n_tiles]
  __half* kp;                        // [N][ld_kp] or null
  float eps, r, ui, ni;
  __device__ void begin(int row) {
    eps = 0.f;
    r = 0.f;
    ui = row < rows ? u[row] : 0.f;
    ni = row < rows ? nrm[row] : 0.f;
  }
  // S^(zeta-1) for one output, zeta fixed at compile time (Z > 0) or general (Z = 0)
  template <int Z>
  __device__ __forceinline__ void run(int col0, const uint32_t* v, uint32_t* out) {
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      float kv[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 c = __ldg(col + col0 + j + h);
        const float S = fmaf(ni * c.y, __uint_as_float(v[j + h]), ui + c.x);
        const float sz1 = Z > 0 ? pow_zm1<Z>(S) : powf(fmaxf(S, 0.f), zeta - 1.f);
        eps = fmaf(c.z, sz1 * S, eps);
        r = fmaf(zeta * c.z, sz1, r);
        kv[h] = c.w * sz1;
      }
      const __half2 h2 = __floats2half2_rn(kv[0], kv[1]);
      out[j / 2] = *reinterpret_cast<const uint32_t*>(&h2);
    }
  }
  // S-dependent sums of one row's 32 columns; out: their 32 FP16 kernel derivatives in pairs
  __device__ __forceinline__ void row_chunk(int col0, const uint32_t* v, uint32_t* out) {
    switch (izeta) {
      case 1: run<1>(col0, v, out); break;
      case 2: run<2>(col0, v, out); break;
      case 3: run<3>(col0, v, out); break;
      case 4: run<4>(col0, v, out); break;
      default: run<0>(col0, v, out); break;
    }
  }
  // The warp's 32 rows (row0 ..) x 32 columns (col0 ..): sums in registers; with kp, the
  // kernel derivatives go to this warp's staging buffer `buf` (64 B per row) and one lane
  // stores the 32 x 32 box with TMA (rows past the end are clipped by the tensor map).
  __device__ void apply_staged(int row, int row0, int col0, const uint32_t* v, unsigned char* stage, int& buf,
                               const CUtensorMap* map) {
    const int lane = threadIdx.x & 31;
    uint32_t out[16];
    if (row < rows) {
      row_chunk(col0, v, out);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) out[k] = 0u;
    }
    if (!kp) return;
    if (lane == 0) bulk_wait_read1();  // the store of two chunks ago has read this buffer
    __syncwarp();
    unsigned char* sb = stage + buf * 2048;
    uint4* dst = reinterpret_cast<uint4*>(sb + lane * 64);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = make_uint4(out[4 * k], out[4 * k + 1], out[4 * k + 2], out[4 * k + 3]);
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) {
      if (row0 < rows) tma_store_2d(map, col0, row0, sb);  // (a box wholly past the end: nothing)
      bulk_commit();
    }
    buf ^= 1;
  }
  __device__ void end(int row, int slot) {
    if (row >= rows) return;
    eps_part[(size_t)row * n_tiles + slot] = eps;
    r_part[(size_t)row * n_tiles + slot] = r;
  }
};

struct EpiGapBwd {
  int rows, d, n_tiles;
  float kappa;
  const float* qbar;    // [Dp]
  const float* r_part;  // [N][n_tiles]
  float* g;             // [N][d]
  float r;
  __device__ void begin(int row) {
    r = 0.f;
    if (row < rows)
      for (int t = 0; t < n_tiles; ++t) r += r_part[(size_t)row * n_tiles + t];
  }
  __device__ void apply(int row, int col0, const uint32_t* v) {
    if (row >= rows) return;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int k = col0 + j;
      if (k < d) g[(size_t)row * d + k] = fmaf(r, __ldg(qbar + k), kappa * __uint_as_float(v[j]));
    }
  }
  __device__ void end(int, int) {}
};

// Kernel rows of the fitting matrices (atoms x sparse set): k(i, s) = S^zeta, and for the
// force rows the weights (w, w S), w = zeta S^(zeta-1) / |p_i|; S as in EpiGapFwd.
struct EpiKernelRows {
  int rows, m, ldw, izeta;
  float zeta;
  const float *u, *nrm, *pnorm;      // [N]
  const float4* col;                 // [Mp] as in EpiGapFwd
  float* k;                          // [N][m]
  float2* wv;                        // [N][ldw] or null
  float ui, ni, ip;
  __device__ void begin(int row) {
    ui = row < rows ? u[row] : 0.f;
    ni = row < rows ? nrm[row] : 0.f;
    ip = (row < rows && wv) ? 1.f / pnorm[row] : 0.f;
  }
  __device__ void apply(int row, int col0, const uint32_t* v) {
    if (row >= rows) return;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int s = col0 + j;
      const float4 c = __ldg(col + s);
      const float S = fmaf(ni * c.y, __uint_as_float(v[j]), ui + c.x);
      float sz1;
      switch (izeta) {
        case 1: sz1 = 1.f; break;
        case 2: sz1 = S; break;
        case 3: sz1 = S * S; break;
        case 4: sz1 = S * S * S; break;
        default: sz1 = powf(fmaxf(S, 0.f), zeta - 1.f); break;
      }
      if (s < m) k[(size_t)row * m + s] = izeta > 0 ? sz1 * S : powf(fmaxf(S, 0.f), zeta);
      if (wv) {
        const float w = zeta * sz1 * ip;
        wv[(size_t)row * ldw + s] = make_float2(w, w * S);
      }
    }
  }
  __device__ void end(int, int) {}
};

// Force rows of the fitting matrices: rows = sparse environments s, columns = projected
// descriptor Jacobian columns J' (see design.cu) ordered by target atom.  With the sparse
// operand [kd (q_s - qbar) | kd | kd] and the column [2^e J' | hi | lo of 2^e qbar.J'], the
// accumulator is kd 2^e q_s.J', and the contribution of a column (owner o, target t,
// component a = col mod 3) is w_os 2^-e / kd times it.  The running sums of one target are
// added to dk[t][a][s] when the target changes (a target's columns are contiguous).
// Tiles of 192 columns are read 24 at a time, so every chunk starts at a column triple (the
// three components of one pair or self slot: one owner, one target, one scale).
struct EpiDesignGrad {
  static constexpr int CHUNK = 24;
  int m, ldw, ncols;
  float inv_kd;
  const int2* col_at;                // [ncols] (owner, target)
  const float4* col_v;               // [ncols] .z = 2^-e of the column's triple
  const float2* wv;                  // [N][ldw] .x = w_os
  float* dk;                         // [N][3][m]
  int target;
  float acc0, acc1, acc2;
  __device__ void flush(int row) {
    if (target >= 0) {
      float* o = dk + (size_t)target * 3 * m + row;
      if (acc0 != 0.f) atomicAdd(o, acc0);
      if (acc1 != 0.f) atomicAdd(o + m, acc1);
      if (acc2 != 0.f) atomicAdd(o + 2 * m, acc2);
    }
    acc0 = acc1 = acc2 = 0.f;
  }
  __device__ void begin(int) {
    target = -1;
    acc0 = acc1 = acc2 = 0.f;
  }
  // Lane 3t reads the record of triple t (coalesced); owner, target and scale reach every
  // lane by shuffles, and the 8 owners' weights at this row are requested before the first
  // use.  All lanes take part (rows past m compute but do not write).
  __device__ void apply(int row, int col0, const uint32_t* v) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool live = row < m;
    const int mine = col0 + lane;
    int2 at_l = make_int2(-1, -1);
    float cz_l = 0.f;
    if (lane < CHUNK && lane % 3 == 0 && mine < ncols) {
      at_l = __ldg(col_at + mine);
      cz_l = __ldg(&col_v[mine].z);
    }
    float wk[CHUNK / 3];
    int tg[CHUNK / 3];
#pragma unroll
    for (int t = 0; t < CHUNK / 3; ++t) {
      const int o = __shfl_sync(FULL, at_l.x, 3 * t);
      const float cz = __shfl_sync(FULL, cz_l, 3 * t);
      tg[t] = __shfl_sync(FULL, at_l.y, 3 * t);
      wk[t] = (live && o >= 0) ? __ldg(&wv[(size_t)o * ldw + row].x) * (cz * inv_kd) : 0.f;
    }
#pragma unroll
    for (int t = 0; t < CHUNK / 3; ++t) {
      if (tg[t] < 0) continue;  // past the last column (same for every lane)
      if (tg[t] != target) {
        if (live) flush(row);
        target = tg[t];
      }
      acc0 = fmaf(wk[t], __uint_as_float(v[3 * t]), acc0);
      acc1 = fmaf(wk[t], __uint_as_float(v[3 * t + 1]), acc1);
      acc2 = fmaf(wk[t], __uint_as_float(v[3 * t + 2]), acc2);
    }
  }
  __device__ void end(int row, int) {
    if (row < m) flush(row);
  }
};

// ------------------------------------------------------------------ the GEMM
// Persistent, warp-specialised: one CTA per SM walks the output tiles (row-major over
// [M/BM] x [N/BN], so CTAs running together share A rows in L2).
//   warp 0, lane 0 : TMA producer, STAGES-deep ring of A/B tiles (full/empty mbarriers)
//   warp 1, lane 0 : MMA issuer, accumulates each tile into one of two TMEM buffers
//   warps 2..      : epilogue, EPI_WARPS warps; warp w reads TMEM lanes 32*(w%4) .. +31 and
//                    a 1/(EPI_WARPS/4) share of the columns; it releases the buffer when done
// so the epilogue of one tile overlaps the MMAs of the next.
// MFAST walks the tiles column-major instead ([N/BN] x [M/BM], m fastest): for a B far
// larger than A, CTAs running together then share B tiles and B is read from memory once.
template <int BN, int STAGES, int EPI_WARPS, class Epi, bool MFAST = false>
__global__ void __launch_bounds__(32 * (2 + EPI_WARPS), 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmC, int num_kb, int m_tiles, int n_tiles, Epi epi, int* err) {
  constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  constexpr int HALVES = EPI_WARPS / 4;           // column groups per tile
  constexpr int COLS = BN / HALVES;               // columns per epilogue warp
  constexpr int CH = EpiChunk<Epi>::value;        // columns per TMEM read
  static_assert((CH == 32 || CH == 24) && COLS % CH == 0, "epilogue chunking");
  // TMEM is allocated in powers of two (>= 32 columns): room for two BN-wide accumulators
  constexpr uint32_t TMEM_COLS = 2 * BN <= 32 ? 32 : 2 * BN <= 64 ? 64 : 2 * BN <= 128 ? 128 : 2 * BN <= 256 ? 256 : 512;
  static_assert(2 * BN <= 512, "two accumulators must fit in tensor memory");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = m_tiles * n_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], EPI_WARPS);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      int issued[STAGES];
      for (int s = 0; s < STAGES; ++s) issued[s] = 0;
      for (int t = blockIdx.x; t < total && !abort_flag; t += gridDim.x) {
        const int m0 = (MFAST ? t % m_tiles : t / n_tiles) * BM, n0 = (MFAST ? t / m_tiles : t % n_tiles) * BN;
        for (int kb = 0; kb < num_kb; ++kb, ++it) {
          const int s = it % STAGES, round = it / STAGES;
          if (round > 0 && !mbar_wait(&empty_bar[s], (round - 1) & 1)) {
            abort_flag = 1;
            break;
          }
          mbar_expect_tx(&full_bar[s], A_BYTES + B_BYTES);
          tma_load_2d(sA + s * A_BYTES, &tmA, kb * BK, m0, &full_bar[s]);
          tma_load_2d(sB + s * B_BYTES, &tmB, kb * BK, n0, &full_bar[s]);
          ++issued[s];
        }
      }
      // every copy started here has landed before the block may exit
      for (int s = 0; s < STAGES; ++s)
        if (issued[s] > 0 && !mbar_wait(&full_bar[s], (issued[s] - 1) & 1)) abort_flag = 1;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(BM, BN);
      int it = 0, lt = 0;
      for (int t = blockIdx.x; t < total && !abort_flag; t += gridDim.x, ++lt) {
        const int b = lt & 1, use = lt >> 1;
        if (use > 0 && !mbar_wait(&tempty_bar[b], (use - 1) & 1)) {
          abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * BN);
        bool ok = true;
        for (int kb = 0; kb < num_kb; ++kb, ++it) {
          const int s = it % STAGES, round = it / STAGES;
          if (!mbar_wait(&full_bar[s], round & 1)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            mma_f16(acc, sw128_desc(a0 + k * 32), sw128_desc(b0 + k * 32), idesc, (kb | k) != 0);
          mma_commit(&empty_bar[s]);
        }
        if (!ok) {
          abort_flag = 1;
          break;
        }
        mma_commit(&tfull_bar[b]);
      }
    }
    __syncwarp();
  } else {
    const int ew = warp - 2;                 // 0 .. EPI_WARPS-1
    const int lg = warp & 3;                 // TMEM lane group this warp may access
    const int half = ew / 4;                 // column group
    unsigned char* stage = sB + STAGES * B_BYTES + ew * 4096;  // staged epilogues only
    int buf = 0;
    int lt = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++lt) {
      const int b = lt & 1, use = lt >> 1;
      const bool ready = __all_sync(0xffffffffu, mbar_wait(&tfull_bar[b], use & 1) && !abort_flag);
      if (!ready) {
        if (lane == 0) {
          abort_flag = 1;
          atomicOr(err, SG_ERR_TIMEOUT);
        }
        break;
      }
      fence_after();
      const int m0 = (MFAST ? t % m_tiles : t / n_tiles) * BM, n0 = (MFAST ? t / m_tiles : t % n_tiles) * BN;
      const int row = m0 + lg * 32 + lane;
      epi.begin(row);
#pragma unroll 1
      for (int c = 0; c < COLS / CH; ++c) {
        uint32_t v[CH];
        const int col = half * COLS + c * CH;
        const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * BN + col);
        if constexpr (CH == 32) {
          tmem_ld32(ta, v);
        } else {
          tmem_ld16_nw(ta, v);
          tmem_ld8_nw(ta + 16, v + 16);
          tmem_wait();
        }
        if constexpr (EpiStaged<Epi>::value) epi.apply_staged(row, m0 + lg * 32, n0 + col, v, stage, buf, &tmC);
        else epi.apply(row, n0 + col, v);
      }
      epi.end(row, (MFAST ? t / m_tiles : t % n_tiles) * HALVES + half);
      fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[b])) : "memory");
    }
    if constexpr (EpiStaged<Epi>::value) {
      if (lane == 0) bulk_wait_all();  // every TMA store of this warp has completed
      __syncwarp();
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
}

template <int BN, int STAGES, int EPI_WARPS = 0, bool STAGED = false>
constexpr size_t smem_bytes() {
  return (size_t)STAGES * (BM * BK * 2 + BN * BK * 2) + 1024 + (STAGED ? (size_t)EPI_WARPS * 4096 : 0);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D FP16 row-major matrix [rows][cols] (cols a multiple of 64) with row stride ld elements
// (ld = cols when 0), tiles of box_rows x 64.
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int box_rows, int ld = 0) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld > 0 ? ld : cols) * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D FP16 output [rows][cols] (row stride cols) written in boxes of 32 x 32 by TMA stores
bool make_store_map(CUtensorMap* m, void* base, int rows, int cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// C = A B^T over K = k; lda, ldb: row strides of A and B in elements (k when 0)
template <int BN, int STAGES, int EPI_WARPS, bool MFAST = false, class Epi>
cudaError_t launch_gemm(const void* A, int a_rows, const void* B, int b_rows, int k, Epi epi, int* err,
                        cudaStream_t st, int lda = 0, int ldb = 0, const CUtensorMap* mc = nullptr) {
  if (k % BK != 0 || a_rows <= 0 || b_rows <= 0) return cudaErrorInvalidValue;
  if ((lda > 0 && lda < k) || (ldb > 0 && ldb < k)) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, a_rows, k, BM, lda) || !make_map(&mb, B, b_rows, k, BN, ldb))
    return cudaErrorInvalidValue;
  auto kern = tc_gemm_kernel<BN, STAGES, EPI_WARPS, Epi, MFAST>;
  constexpr size_t smem = smem_bytes<BN, STAGES, EPI_WARPS, EpiStaged<Epi>::value>();
  static_assert(smem <= 227 * 1024, "shared memory per block");
  cudaError_t e = sg_set_smem<tc_gemm_kernel<BN, STAGES, EPI_WARPS, Epi, MFAST>>(smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int m_tiles = (a_rows + BM - 1) / BM, n_tiles = (b_rows + BN - 1) / BN;
  if ((long long)m_tiles * n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = std::min(sms, m_tiles * n_tiles);
  kern<<<grid, 32 * (2 + EPI_WARPS), smem, st>>>(ma, mb, mc ? *mc : ma, k / BK, m_tiles, n_tiles, epi, err);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ operand preparation
// one warp per atom: u = (q - qbar)/|q - qbar| in FP16, A row = [hi] (TERMS = 1, row
// stride dp) or the split [hi | hi | lo] (TERMS = 3, row stride 3 dp)
template <int TERMS>
__global__ void prep_atoms_kernel(const float* __restrict__ q, int n, int d, int dp,
                                  const float* __restrict__ qbar, __half* A, float* nrm, float* uq) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const float* qi = q + (size_t)i * d;
  float ss = 0.f, dq = 0.f;
  for (int k = lane; k < d; k += 32) {
    const float t = qi[k] - qbar[k];
    ss = fmaf(t, t, ss);
    dq = fmaf(t, qbar[k], dq);
  }
  ss = warp_sum(ss);
  dq = warp_sum(dq);
  const float nn = sqrtf(ss);
  const float inv = nn > 0.f ? 1.f / nn : 0.f;
  __half* row = A + (size_t)i * TERMS * dp;
  for (int k = lane; k < dp; k += 32) {
    const float uk = k < d ? (qi[k] - qbar[k]) * inv : 0.f;
    const __half hi = __float2half_rn(uk);
    row[k] = hi;
    if (TERMS == 3) {
      row[dp + k] = hi;
      row[2 * dp + k] = __float2half_rn(uk - __half2float(hi));
    }
  }
  if (lane == 0) {
    nrm[i] = nn;
    uq[i] = dq;
  }
}

}  // namespace

// Tile configurations of the two GAP products, chosen by the autotuner.  Each is a
// (columns per tile BN, pipeline stages, epilogue warps) instance of tc_gemm_kernel:
//   forward  0: (256, 4, 8)   1: (128, 6, 4)   2: (128, 6, 8)
//   backward 0: (224, 5, 4)   1: (128, 6, 4)   2: (192, 5, 4)   3: (256, 4, 4)   4: (160, 6, 4)
// The forward's columns are the sparse set padded to 256 (every BN above divides it); the
// backward's, the descriptor padded to 64 (ragged last tiles read TMA's zero fill).
static int fwd_bn(int cfg) { return cfg == 0 ? 256 : 128; }
static int fwd_halves(int cfg) { return cfg == 1 ? 1 : 2; }

// partial-sum slots per row of the forward epilogue: one per column group of every tile
int sg_gap_tc_tiles(int mp, int fwd_cfg) { return mp / fwd_bn(fwd_cfg) * fwd_halves(fwd_cfg); }
int sg_gap_tc_tiles_max(int mp) { return mp / 64; }

cudaError_t sg_gap_tc_prepare(const float* q, int n, int d, int dp, const float* qbar, __half* A, float* nrm,
                              float* uq, int terms, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (terms == 1)
    prep_atoms_kernel<1><<<(n * 32 + 127) / 128, 128, 0, st>>>(q, n, d, dp, qbar, A, nrm, uq);
  else if (terms == 3)
    prep_atoms_kernel<3><<<(n * 32 + 127) / 128, 128, 0, st>>>(q, n, d, dp, qbar, A, nrm, uq);
  else
    return cudaErrorInvalidValue;
  ++sg_kernel_launches;
  return cudaGetLastError();
}

cudaError_t sg_gap_tc_forward(const GapTcModel& md, int terms, const __half* A, const float* nrm,
                              const float* uq, int n, float* eps_part, float* r_part, __half* kp, int* err,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (terms != 1 && terms != 3) return cudaErrorInvalidValue;
  EpiGapFwd e{};
  e.rows = n;
  e.ld_kp = md.mp;
  e.n_tiles = sg_gap_tc_tiles(md.mp, md.fwd_cfg);
  e.izeta = md.izeta;
  e.zeta = md.zeta;
  e.u = uq;
  e.nrm = nrm;
  e.col = md.col;
  e.eps_part = eps_part;
  e.r_part = r_part;
  e.kp = kp;
  // one FP16 product hi.hi: A rows [hi] against the first dp columns of the sparse rows
  // [hi | lo | hi]; three: A rows [hi | hi | lo] against the whole rows
  const int k = terms * md.dp, lda = terms * md.dp, ldb = 3 * md.dp;
  // the kernel derivatives [n][mp] leave through shared memory in 32 x 32 TMA stores
  CUtensorMap mc;
  if (kp && !make_store_map(&mc, kp, n, md.mp)) return cudaErrorInvalidValue;
  const CUtensorMap* pmc = kp ? &mc : nullptr;
  switch (md.fwd_cfg) {
    case 0: return launch_gemm<256, 4, 8>(A, n, md.B, md.mp, k, e, err, st, lda, ldb, pmc);
    case 1: return launch_gemm<128, 6, 4>(A, n, md.B, md.mp, k, e, err, st, lda, ldb, pmc);
    case 2: return launch_gemm<128, 6, 8>(A, n, md.B, md.mp, k, e, err, st, lda, ldb, pmc);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t sg_gap_tc_backward(const GapTcModel& md, const __half* kp, const float* r_part, int n, float* g,
                               int* err, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  EpiGapBwd e{};
  e.rows = n;
  e.d = md.d;
  e.n_tiles = sg_gap_tc_tiles(md.mp, md.fwd_cfg);  // the forward's partial-sum layout
  e.kappa = md.kappa;
  e.qbar = md.qbar;
  e.r_part = r_part;
  e.g = g;
  switch (md.bwd_cfg) {
    case 0: return launch_gemm<224, 5, 4>(kp, n, md.BT, md.dp, md.mp, e, err, st);
    case 1: return launch_gemm<128, 6, 4>(kp, n, md.BT, md.dp, md.mp, e, err, st);
    case 2: return launch_gemm<192, 5, 4>(kp, n, md.BT, md.dp, md.mp, e, err, st);
    case 3: return launch_gemm<256, 4, 4>(kp, n, md.BT, md.dp, md.mp, e, err, st);
    case 4: return launch_gemm<160, 6, 4>(kp, n, md.BT, md.dp, md.mp, e, err, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t sg_tc_gemm_store(const __half* A, int m, const __half* B, int nn, int k, float* C, int* err,
                             cudaStream_t st) {
  EpiStore e{m, nn, C};
  return launch_gemm<128, 6, 4>(A, m, B, nn, k, e, err, st);
}

cudaError_t sg_tc_kernel_rows(const GapTcModel& md, const __half* A, const float* nrm, const float* uq, int n,
                              int m, const float* pnorm, float* k, float2* wv, int* err, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  EpiKernelRows e{};
  e.rows = n;
  e.m = m;
  e.ldw = md.mp;
  e.izeta = md.izeta;
  e.zeta = md.zeta;
  e.u = uq;
  e.nrm = nrm;
  e.pnorm = pnorm;
  e.col = md.col;
  e.k = k;
  e.wv = wv;
  return launch_gemm<256, 4, 8>(A, n, md.B, md.mp, 3 * md.dp, e, err, st);
}

cudaError_t sg_tc_design_grad(const GapTcModel& md, int m, const __half* J, long long ncols, const int2* col_at,
                              const float4* col_v, const float2* wv, float* dk, int* err, cudaStream_t st) {
  if (ncols == 0) return cudaSuccess;
  if (ncols > 0x7fffffffLL - 256) return cudaErrorInvalidValue;
  EpiDesignGrad e{};
  e.m = m;
  e.ldw = md.mp;
  e.ncols = (int)ncols;
  e.inv_kd = 1.f / md.kd;
  e.col_at = col_at;
  e.col_v = col_v;
  e.wv = wv;
  e.dk = dk;
  // A = the scaled centred sparse rows with their two unit columns, K = dpd
  return launch_gemm<192, 5, 16, true>(md.Ad, md.mp, J, (int)ncols, md.dpd, e, err, st);
}
