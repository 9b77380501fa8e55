// Cell-list neighbour builder, bit-exact against a brute-force FP64 search.
//
// A pair (i, j, S) is kept when |x_j + S.h - x_i|^2 < r_cut^2, evaluated in FP64 with
// one fixed operation order and no contraction into FMA:
//   s = (S1*h1 + S2*h2) + S3*h3,  r = (x_j + s) - x_i  in canonical orientation
//   (i < j, or i == j with S lexicographically positive), r = -((x_i + (-s)) - x_j)
//   otherwise, d2 = (rx*rx + ry*ry) + rz*rz.
// The canonical orientation makes the set exactly symmetric ((j, i, -S) is kept with
// r_ji = -r_ij bit for bit), which the deterministic force gather relies on.
// Candidates come from bins laid out in fractional coordinates; an FP32 distance decides
// every candidate whose d2 is farther than a rigorous rounding margin from r_cut^2 (or
// from 0), and the FP64 expression decides the rest, so the set equals the FP64 one.
// Pairs of each (centre, neighbour species) segment are sorted by (j, S).
#include <algorithm>

#include "internal.h"

// ---------------------------------------------------------------- scan
#define SCAN_BLOCK 1024
size_t sg_scan_tmp_ints(int n) { return (size_t)(n + SCAN_BLOCK - 1) / SCAN_BLOCK + 1; }

__global__ void scan_block_sums(const int* in, int n, int* sums, const int* run) {
  if (run && *run == 0) return;
  __shared__ int sh[32];
  int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int v = 0;
  for (int k = 0; k < SCAN_BLOCK / 256; ++k) {
    int idx = blockIdx.x * SCAN_BLOCK + k * 256 + threadIdx.x;
    if (idx < n) v += in[idx];
  }
  (void)i;
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int w = threadIdx.x < 8 ? sh[threadIdx.x] : 0;
    w = warp_sum(w);
    if (threadIdx.x == 0) sums[blockIdx.x] = w;
  }
}

// single block: exclusive scan of the block sums in place (nb <= a few thousand)
__global__ void scan_sums(int* sums, int nb, const int* run) {
  if (run && *run == 0) return;
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    int idx = base + threadIdx.x;
    int v = idx < nb ? sums[idx] : 0;
    // block inclusive scan
    __shared__ int sh[1024];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    int incl = sh[threadIdx.x];
    int c = carry;
    if (idx < nb) sums[idx] = c + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_apply(const int* in, int* out, int n, const int* sums, const int* run) {
  if (run && *run == 0) return;
  __shared__ int sh[SCAN_BLOCK];
  const int base = blockIdx.x * SCAN_BLOCK;
  for (int k = threadIdx.x; k < SCAN_BLOCK; k += blockDim.x) sh[k] = (base + k < n) ? in[base + k] : 0;
  __syncthreads();
  // per-thread sequential chunk of 4, then a block scan of chunk totals
  const int t = threadIdx.x;  // 256 threads, 4 items each
  int v0 = sh[4 * t], v1 = sh[4 * t + 1], v2 = sh[4 * t + 2], v3 = sh[4 * t + 3];
  int tot = v0 + v1 + v2 + v3;
  __shared__ int ts[256];
  ts[t] = tot;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    int x = t >= o ? ts[t - o] : 0;
    __syncthreads();
    ts[t] += x;
    __syncthreads();
  }
  int excl = ts[t] - tot + sums[blockIdx.x];
  int idx = base + 4 * t;
  if (idx < n) out[idx] = excl;
  if (idx + 1 < n) out[idx + 1] = excl + v0;
  if (idx + 2 < n) out[idx + 2] = excl + v0 + v1;
  if (idx + 3 < n) out[idx + 3] = excl + v0 + v1 + v2;
  if (blockIdx.x == gridDim.x - 1 && t == 255) out[n] = sums[gridDim.x];
}

// out[0..n] = exclusive scan of in[0..n-1], out[n] = total.  tmp: sg_scan_tmp_ints(n) ints.
cudaError_t sg_exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t st,
                              const int* run) {
  if (n <= 0) {
    if (!run) cudaMemsetAsync(out, 0, sizeof(int), st);
    return cudaGetLastError();
  }
  const int nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  scan_block_sums<<<nb, 256, 0, st>>>(in, n, tmp, run);
  scan_sums<<<1, 1024, 0, st>>>(tmp, nb, run);
  scan_apply<<<nb, 256, 0, st>>>(in, out, n, tmp, run);
  sg_kernel_launches += 3;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- binning
__global__ void bin_assign(const double* __restrict__ pos, int n, NbrBuffers b) {
  if (b.run && *b.run == 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const StructGeom& g = b.geom[b.atom_struct[i]];
  double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  int bi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double f = x * g.hinv[k] + y * g.hinv[3 + k] + z * g.hinv[6 + k];
    f = f * g.nb[k];
    int c = (f >= 0.0) ? (f < (double)g.nb[k] ? (int)f : g.nb[k] - 1) : 0;
    bi[k] = c;
  }
  int id = g.bin_off + (bi[0] * g.nb[1] + bi[1]) * g.nb[2] + bi[2];
  b.atom_bin[i] = id;
  b.atom_bin4[i] = make_int4(bi[0], bi[1], bi[2], id);
  b.atom_slot[i] = atomicAdd(&b.bin_count[id], 1);
}

// binpos[.].w packs the atom index (bits 0..27) and its species (bits 28..30), so the
// candidate sweep needs no second dependent load for the species of a kept neighbour
__global__ void bin_fill(const double* __restrict__ pos, const int* __restrict__ species, int n, NbrBuffers b,
                         float4* binpos) {
  if (b.run && *b.run == 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int at = b.bin_start[b.atom_bin[i]] + b.atom_slot[i];
  b.bin_atoms[at] = i;
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  const float xh = (float)x, yh = (float)y, zh = (float)z;
  const float4 lo = make_float4((float)(x - (double)xh), (float)(y - (double)yh), (float)(z - (double)zh), 0.f);
  binpos[at] = make_float4(xh, yh, zh, __int_as_float(i | (species[i] << 28)));
  b.atom_hi[i] = make_float4(xh, yh, zh, 0.f);
  b.atom_lo[i] = lo;
}

__global__ void wrap_kernel(const double* __restrict__ pos, int n, NbrBuffers b, double* pos_w,
                            int4* img) {
  if (b.run && *b.run == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const StructGeom& g = b.geom[b.atom_struct[i]];
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  double nk[3];
  bool moved = false, finite = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double f = x * g.hinv[k] + y * g.hinv[3 + k] + z * g.hinv[6 + k];
    finite &= isfinite(f);
    nk[k] = (f >= -1e-9 && f < 1.0 + 1e-9) ? 0.0 : floor(f);
    moved |= nk[k] != 0.0;
  }
  if (!finite) {
    atomicOr(b.err, SG_ERR_OUTSIDE_CELL);
    nk[0] = nk[1] = nk[2] = 0.0;
    moved = false;
  }
  double w[3] = {x, y, z};
  if (moved) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      w[c] = __dsub_rn(w[c], __dadd_rn(__dadd_rn(__dmul_rn(nk[0], g.h[c]), __dmul_rn(nk[1], g.h[3 + c])),
                                        __dmul_rn(nk[2], g.h[6 + c])));
  }
  pos_w[3 * i] = w[0];
  pos_w[3 * i + 1] = w[1];
  pos_w[3 * i + 2] = w[2];
  img[i] = make_int4((int)nk[0], (int)nk[1], (int)nk[2], 0);
}

cudaError_t sg_nbr_wrap(const double* pos, int n_atoms, const NbrBuffers& b, double* pos_w,
                        int4* img, cudaStream_t st) {
  if (n_atoms > 0) {
    wrap_kernel<<<(n_atoms + 255) / 256, 256, 0, st>>>(pos, n_atoms, b, pos_w, img);
    ++sg_kernel_launches;
  }
  return cudaGetLastError();
}

cudaError_t sg_nbr_bin(const double* pos, const int* species, int n_atoms, int n_bins, const NbrBuffers& b,
                       cudaStream_t st) {
  cudaMemsetAsync(b.bin_count, 0, sizeof(int) * (size_t)n_bins, st);
  if (n_atoms > 0) {
    bin_assign<<<(n_atoms + 255) / 256, 256, 0, st>>>(pos, n_atoms, b);
    ++sg_kernel_launches;
  }
  cudaError_t e = sg_exclusive_scan(b.bin_count, b.bin_start, n_bins, b.scan_tmp, st, b.run);
  if (e != cudaSuccess) return e;
  if (n_atoms > 0) {
    bin_fill<<<(n_atoms + 255) / 256, 256, 0, st>>>(pos, species, n_atoms, b, b.binpos);
    ++sg_kernel_launches;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pair search
__device__ __forceinline__ bool lex_positive(int s1, int s2, int s3) {
  return s1 > 0 || (s1 == 0 && (s2 > 0 || (s2 == 0 && s3 > 0)));
}

// ---- double-float (hi + lo FP32) arithmetic, exact error terms by TwoSum / TwoProd
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (a_hi + a_lo) + (b_hi + b_lo), renormalised
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  two_sum(s, e, sh, sl);
}
// image shift S.h in double-float from the split lattice vectors (S integer, |S| < 2^8)
__device__ __forceinline__ void df_shift(const StructGeom& g, float f1, float f2, float f3, int c, float& sh,
                                         float& sl) {
  float ph = __fmul_rn(f1, g.h32[c]), pl = __fmaf_rn(f1, g.h32[c], -ph);  // exact product
  pl = __fmaf_rn(f1, g.h32lo[c], pl);
  float qh = __fmul_rn(f2, g.h32[3 + c]), ql = __fmaf_rn(f2, g.h32[3 + c], -qh);
  ql = __fmaf_rn(f2, g.h32lo[3 + c], ql);
  float rh = __fmul_rn(f3, g.h32[6 + c]), rl = __fmaf_rn(f3, g.h32[6 + c], -rh);
  rl = __fmaf_rn(f3, g.h32lo[6 + c], rl);
  float th, tl;
  df_add(ph, pl, qh, ql, th, tl);
  df_add(th, tl, rh, rl, sh, sl);
}

// bin coordinate t (possibly outside [0, n)) -> periodic bin and image index, no division
__device__ __forceinline__ void wrap(int t, int n, int& bin, int& S, float& Sf) {
  S = 0;
  while (t < 0) { t += n; --S; }
  while (t >= n) { t -= n; ++S; }
  bin = t;
  Sf = (float)S;
}

// exact FP64 separation (fixed operation order, no FMA) in canonical orientation, from the
// FP64 shift s = (S1*h1 + S2*h2) + S3*h3
__device__ __forceinline__ void exact_sep(const double* __restrict__ pos, int i, int j, const double s[3],
                                         bool canon, double r[3], double& d2) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double xi = pos[3 * i + c], xj = pos[3 * j + c];
    r[c] = canon ? __dsub_rn(__dadd_rn(xj, s[c]), xi) : -__dsub_rn(__dadd_rn(xi, -s[c]), xj);
  }
  d2 = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])), __dmul_rn(r[2], r[2]));
}

// Visit every kept pair of atom i; lanes of the warp take candidates in parallel.
// fn(lane_has_pair, j, k, S1, S2, S3, f1, f2, f3, s[3], r[3], d2) is called by all lanes
// together (k: the candidate's slot in bin order, f = (float)S), with the
// FP64 shift s of this image; d2 < 0 marks a pair kept by the FP32 test whose exact FP64
// separation has not been computed.  The FP32 test uses FP32 positions and the FP32
// lattice vectors; the rounding margin covers both.  FP64 work (slow on this GPU) is done
// only where needed: the shift once per image by one lane, separations for kept pairs.
template <typename Fn>
__device__ __forceinline__ void visit_pairs(const double* __restrict__ pos, const float4* binpos,
                                            int i, double rc, const NbrBuffers& b, Fn&& fn) {
  const int lane = threadIdx.x & 31;
  const StructGeom& g = b.geom[b.atom_struct[i]];
  const double rc2 = rc * rc;
  const float rc2f = (float)rc2;
  const float margin = g.margin;
  const float xi = (float)pos[3 * i], yi = (float)pos[3 * i + 1], zi = (float)pos[3 * i + 2];
  const int4 cb = b.atom_bin4[i];
  for (int d0 = -g.m[0]; d0 <= g.m[0]; ++d0) {
    int b0, S1;
    float f1;
    wrap(cb.x + d0, g.nb[0], b0, S1, f1);
    for (int d1 = -g.m[1]; d1 <= g.m[1]; ++d1) {
      int b1, S2;
      float f2;
      wrap(cb.y + d1, g.nb[1], b1, S2, f2);
      // bins cb.z - m .. cb.z + m are contiguous in bin order within one z-image: sweep
      // each image's run of bins as one candidate range
      const int zlo = cb.z - g.m[2], zhi = cb.z + g.m[2];
      int S3 = 0, t0 = zlo;
      while (t0 < 0) { t0 += g.nb[2]; --S3; }
      while (t0 >= g.nb[2]) { t0 -= g.nb[2]; ++S3; }
      for (int t = zlo; t <= zhi; ++S3, t0 = 0) {
        // run: z-bins t0 .. t1 of image S3, covering t .. t + (t1 - t0)
        const int t1 = min(g.nb[2] - 1, t0 + (zhi - t));
        t += t1 - t0 + 1;
        const float f3 = (float)S3;
        const float sx = __fadd_rn(__fadd_rn(__fmul_rn(f1, g.h32[0]), __fmul_rn(f2, g.h32[3])), __fmul_rn(f3, g.h32[6]));
        const float sy = __fadd_rn(__fadd_rn(__fmul_rn(f1, g.h32[1]), __fmul_rn(f2, g.h32[4])), __fmul_rn(f3, g.h32[7]));
        const float sz = __fadd_rn(__fadd_rn(__fmul_rn(f1, g.h32[2]), __fmul_rn(f2, g.h32[5])), __fmul_rn(f3, g.h32[8]));
        const int tb = g.bin_off + (b0 * g.nb[1] + b1) * g.nb[2];
        const int beg = b.bin_start[tb + t0], end = b.bin_start[tb + t1 + 1];
        const bool zero_shift = (S1 == 0 && S2 == 0 && S3 == 0);
        const bool lexpos = lex_positive(S1, S2, S3);
        double s[3] = {0.0, 0.0, 0.0};
        bool have_s = false;
        // two candidates per lane and step: both position loads are in flight together
        auto test = [&](int k, int& j, int& sj, bool& cand, bool& exact) {
          j = -1;
          sj = 0;
          cand = exact = false;
          if (k < end) {
            const float4 pj = binpos[k];
            const int w = __float_as_int(pj.w);
            j = w & 0x0FFFFFFF;
            sj = w >> 28;
            if (!(j == i && zero_shift)) {
              // explicit round-to-nearest ops: the count and fill kernels decide alike
              const float dx = __fsub_rn(__fadd_rn(pj.x, sx), xi);
              const float dy = __fsub_rn(__fadd_rn(pj.y, sy), yi);
              const float dz = __fsub_rn(__fadd_rn(pj.z, sz), zi);
              const float d2f = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
              exact = fabsf(d2f - rc2f) <= margin || d2f <= margin;
              cand = exact || d2f < rc2f;
            }
          }
        };
        auto decide = [&](int j, int sj, bool cand, bool exact) {
          bool keep = false;
          double r[3] = {0, 0, 0}, d2 = -1.0;
          if (cand) {
            if (exact) {
              const bool canon = (j > i) || (j == i && lexpos);
              exact_sep(pos, i, j, s, canon, r, d2);
              keep = d2 < rc2;
              if (keep && d2 == 0.0) atomicOr(b.err, SG_ERR_COINCIDENT);
            } else {
              keep = true;  // exact value computed on demand by the caller
            }
          }
          fn(keep, j, sj, S1, S2, S3, f1, f2, f3, s, r, d2);
        };
        for (int base = beg; base < end; base += 64) {
          int ja, sja, jb, sjb;
          bool ca, ea, cb, eb;
          test(base + lane, ja, sja, ca, ea);
          test(base + 32 + lane, jb, sjb, cb, eb);
          if (!have_s && __any_sync(0xffffffffu, ea || eb || ((ca || cb) && Fn::kNeedsShift))) {
            if (lane == 0) {
#pragma unroll
              for (int c = 0; c < 3; ++c)
                s[c] = __dadd_rn(__dadd_rn(__dmul_rn((double)S1, g.h[c]), __dmul_rn((double)S2, g.h[3 + c])),
                                 __dmul_rn((double)S3, g.h[6 + c]));
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) s[c] = __shfl_sync(0xffffffffu, s[c], 0);
            have_s = true;
          }
          decide(ja, sja, ca, ea);
          if (base + 32 < end) decide(jb, sjb, cb, eb);
        }
      }
    }
  }
}

__device__ __forceinline__ unsigned long long pair_key(int j, int s1, int s2, int s3) {
  return ((unsigned long long)(unsigned)j << 24) | ((unsigned long long)(s1 + 128) << 16) |
         ((unsigned long long)(s2 + 128) << 8) | (unsigned long long)(s3 + 128);
}

// One sweep over the candidates of atom i: each kept pair's key goes to the atom's slot
// array (in visit order), and the kept pairs are counted per neighbour species.
struct FillSlots {
  static constexpr bool kNeedsShift = false;
  int lane, maxn;
  int* cnt;                      // running slot count (warp-uniform)
  int* percnt;                   // per-lane counts by species [SG_MAX_SPECIES]
  unsigned long long* slots;     // this atom's maxn slots
  int* err;
  __device__ void operator()(bool keep, int j, int sj, int S1, int S2, int S3, float, float, float,
                             const double*, const double*, double) const {
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (keep) {
#pragma unroll
      for (int s = 0; s < SG_MAX_SPECIES; ++s) percnt[s] += (s == sj);
      const int at = *cnt + __popc(mask & ((1u << lane) - 1u));
      if (at < maxn) slots[at] = pair_key(j, S1, S2, S3);
      else atomicOr(err, SG_ERR_PAIR_CAPACITY);
    }
    *cnt += __popc(mask);
  }
};

__global__ void fill_slots_kernel(const double* __restrict__ pos, const int* __restrict__ species,
                                  int n, int nsp, double rc, int maxn, NbrBuffers b,
                                  const float4* binpos) {
  if (b.run && *b.run == 0) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int i = warp;
  int cnt = 0;
  int percnt[SG_MAX_SPECIES];
#pragma unroll
  for (int s = 0; s < SG_MAX_SPECIES; ++s) percnt[s] = 0;
  visit_pairs(pos, binpos, i, rc, b,
              FillSlots{lane, maxn, &cnt, percnt, b.key_tmp + (size_t)i * maxn, b.err});
  for (int s = 0; s < nsp; ++s) {
    const int v = warp_sum(percnt[s]);
    if (lane == 0) b.seg_count[i * nsp + s] = v;
  }
  if (lane == 0) {
    b.slot_count[i] = cnt;
    atomicMax(b.max_count, cnt);
  }
}

// ---- the same sweep organised by bin
// One block per bin (persistent over bins): the candidates of the bin's neighbour bins, in
// every periodic image, are staged once in shared memory with their FP32 image shift already
// added (the same rounded sums as visit_pairs, so every decision is bit-identical), and each
// centre atom of the bin, one warp each, tests them there.  The bin's atoms share the 27 (or
// more) neighbour bins, so the candidates are read from memory once per bin instead of once
// per atom.  A bin whose neighbourhood has more than NB_CAP candidates, more than NB_COLS
// (x, y) bin columns or more than NB_RPC z-runs per column (small cells with many images)
// takes the per-atom sweep instead.
constexpr int NB_WARPS = 4;
constexpr int NB_CAP = 1536;   // candidates staged per bin
constexpr int NB_COLS = 32;    // (x, y) bin columns of a bin's neighbourhood
constexpr int NB_RPC = 4;      // z-runs per column

__device__ __forceinline__ int pack_shift(int s1, int s2, int s3) {
  return ((s1 + 128) << 16) | ((s2 + 128) << 8) | (s3 + 128);
}

__global__ void __launch_bounds__(NB_WARPS * 32)
fill_slots_bins_kernel(const double* __restrict__ pos, int nsp, double rc, int maxn, NbrBuffers b,
                       const float4* __restrict__ binpos) {
  if (b.run && *b.run == 0) return;
  __shared__ float4 cpos[NB_CAP];      // candidate position + image shift, .w = j | species << 28
  __shared__ int cshift[NB_CAP];       // candidate image S, packed
  __shared__ int run_beg[NB_COLS * NB_RPC], run_len[NB_COLS * NB_RPC], run_S[NB_COLS * NB_RPC];
  __shared__ float run_sx[NB_COLS * NB_RPC], run_sy[NB_COLS * NB_RPC], run_sz[NB_COLS * NB_RPC];
  __shared__ int run_off[NB_COLS * NB_RPC + 1];
  __shared__ int col_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double rc2 = rc * rc;
  const float rc2f = (float)rc2;
  for (int bin = blockIdx.x; bin < b.n_bins; bin += gridDim.x) {
    const int a_beg = b.bin_start[bin], a_end = b.bin_start[bin + 1];
    if (a_beg == a_end) continue;  // no centre atom (the same for the whole block)
    // structure of this bin: the last s with bin_off <= bin (every structure has a bin)
    int lo = 0, hi = b.n_struct - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.geom[mid].bin_off <= bin) lo = mid;
      else hi = mid - 1;
    }
    const StructGeom& g = b.geom[lo];
    const int local = bin - g.bin_off;
    const int bx = local / (g.nb[1] * g.nb[2]), by = (local / g.nb[2]) % g.nb[1], bz = local % g.nb[2];
    const int ncols = (2 * g.m[0] + 1) * (2 * g.m[1] + 1);
    __syncthreads();  // the previous bin's candidates are no longer read
    if (tid == 0) col_ok = ncols <= NB_COLS;
    __syncthreads();
    // ---- runs: thread t < ncols walks column t = (d0, d1) and its z-runs (as visit_pairs)
    if (col_ok && tid < NB_COLS) {
      int nr = 0;
      if (tid < ncols) {
        const int d0 = tid / (2 * g.m[1] + 1) - g.m[0], d1 = tid % (2 * g.m[1] + 1) - g.m[1];
        int b0, S1, b1, S2;
        float f1, f2;
        wrap(bx + d0, g.nb[0], b0, S1, f1);
        wrap(by + d1, g.nb[1], b1, S2, f2);
        const int zlo = bz - g.m[2], zhi = bz + g.m[2];
        int S3 = 0, t0 = zlo;
        while (t0 < 0) { t0 += g.nb[2]; --S3; }
        while (t0 >= g.nb[2]) { t0 -= g.nb[2]; ++S3; }
        const int tb = g.bin_off + (b0 * g.nb[1] + b1) * g.nb[2];
        for (int t = zlo; t <= zhi; ++S3, t0 = 0) {
          const int t1 = min(g.nb[2] - 1, t0 + (zhi - t));
          t += t1 - t0 + 1;
          const int beg = b.bin_start[tb + t0], end = b.bin_start[tb + t1 + 1];
          if (end > beg) {
            if (nr == NB_RPC) {
              nr = NB_RPC + 1;  // too many runs in this column
              break;
            }
            const int k = tid * NB_RPC + nr;
            const float f3 = (float)S3;
            run_beg[k] = beg;
            run_len[k] = end - beg;
            run_S[k] = pack_shift(S1, S2, S3);
            run_sx[k] = __fadd_rn(__fadd_rn(__fmul_rn(f1, g.h32[0]), __fmul_rn(f2, g.h32[3])), __fmul_rn(f3, g.h32[6]));
            run_sy[k] = __fadd_rn(__fadd_rn(__fmul_rn(f1, g.h32[1]), __fmul_rn(f2, g.h32[4])), __fmul_rn(f3, g.h32[7]));
            run_sz[k] = __fadd_rn(__fadd_rn(__fmul_rn(f1, g.h32[2]), __fmul_rn(f2, g.h32[5])), __fmul_rn(f3, g.h32[8]));
            ++nr;
          }
        }
      }
      // empty run slots of the column, then candidate offsets of all runs (warp 0 scan)
      for (int r = min(nr, NB_RPC); r < NB_RPC; ++r) run_len[tid * NB_RPC + r] = 0;
      const bool bad = nr > NB_RPC;
      int cnt = 0;
      for (int r = 0; r < NB_RPC; ++r) cnt += run_len[tid * NB_RPC + r];
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      int off = incl - cnt;
      for (int r = 0; r < NB_RPC; ++r) {
        run_off[tid * NB_RPC + r] = off;
        off += run_len[tid * NB_RPC + r];
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      if (tid == 31) run_off[NB_COLS * NB_RPC] = total;
      if (__any_sync(0xffffffffu, bad) || total > NB_CAP) {
        if (tid == 0) col_ok = 0;
      }
    }
    __syncthreads();
    const bool staged = col_ok != 0;
    if (staged) {
      const int total = run_off[NB_COLS * NB_RPC];
      for (int c = tid; c < total; c += NB_WARPS * 32) {
        int rlo = 0, rhi = NB_COLS * NB_RPC - 1;  // the last run with run_off <= c and run_len > 0
        while (rlo < rhi) {
          const int mid = (rlo + rhi + 1) >> 1;
          if (run_off[mid] <= c) rlo = mid;
          else rhi = mid - 1;
        }
        while (run_len[rlo] == 0 || run_off[rlo] + run_len[rlo] <= c) ++rlo;  // skip empty slots
        const float4 pj = binpos[run_beg[rlo] + (c - run_off[rlo])];
        cpos[c] = make_float4(__fadd_rn(pj.x, run_sx[rlo]), __fadd_rn(pj.y, run_sy[rlo]),
                              __fadd_rn(pj.z, run_sz[rlo]), pj.w);
        cshift[c] = run_S[rlo];
      }
    }
    __syncthreads();
    const int total = staged ? run_off[NB_COLS * NB_RPC] : 0;
    // ---- centre atoms of the bin, one warp each
    for (int ca = a_beg + warp; ca < a_end; ca += NB_WARPS) {
      const int i = b.bin_atoms[ca];
      int cnt = 0;
      int percnt[SG_MAX_SPECIES];
#pragma unroll
      for (int s = 0; s < SG_MAX_SPECIES; ++s) percnt[s] = 0;
      FillSlots fn{lane, maxn, &cnt, percnt, b.key_tmp + (size_t)i * maxn, b.err};
      if (!staged) {
        visit_pairs(pos, binpos, i, rc, b, FillSlots(fn));  // (a copy: it refers to cnt and percnt)
      } else {
        const float xi = (float)pos[3 * i], yi = (float)pos[3 * i + 1], zi = (float)pos[3 * i + 2];
        const float margin = g.margin;
        const int zero = pack_shift(0, 0, 0);
        auto test = [&](int k, int& j, int& sj, int& S, bool& cand, bool& exact) {
          j = -1;
          sj = 0;
          S = zero;
          cand = exact = false;
          if (k < total) {
            const float4 pj = cpos[k];
            const int w = __float_as_int(pj.w);
            j = w & 0x0FFFFFFF;
            sj = w >> 28;
            S = cshift[k];
            if (!(j == i && S == zero)) {
              // explicit round-to-nearest ops, as visit_pairs (the shift is already in pj)
              const float dx = __fsub_rn(pj.x, xi);
              const float dy = __fsub_rn(pj.y, yi);
              const float dz = __fsub_rn(pj.z, zi);
              const float d2f = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
              exact = fabsf(d2f - rc2f) <= margin || d2f <= margin;
              cand = exact || d2f < rc2f;
            }
          }
        };
        auto decide = [&](int j, int sj, int S, bool cand, bool exact) {
          const int S1 = ((S >> 16) & 255) - 128, S2 = ((S >> 8) & 255) - 128, S3 = (S & 255) - 128;
          bool keep = false;
          double r[3] = {0, 0, 0}, d2 = -1.0, sh[3] = {0, 0, 0};
          if (cand) {
            if (exact) {
#pragma unroll
              for (int c = 0; c < 3; ++c)
                sh[c] = __dadd_rn(__dadd_rn(__dmul_rn((double)S1, g.h[c]), __dmul_rn((double)S2, g.h[3 + c])),
                                  __dmul_rn((double)S3, g.h[6 + c]));
              const bool canon = (j > i) || (j == i && lex_positive(S1, S2, S3));
              exact_sep(pos, i, j, sh, canon, r, d2);
              keep = d2 < rc2;
              if (keep && d2 == 0.0) atomicOr(b.err, SG_ERR_COINCIDENT);
            } else {
              keep = true;
            }
          }
          fn(keep, j, sj, S1, S2, S3, 0.f, 0.f, 0.f, sh, r, d2);
        };
        for (int base = 0; base < total; base += 64) {
          int ja, sja, Sa, jb, sjb, Sb;
          bool ca_, ea, cb, eb;
          test(base + lane, ja, sja, Sa, ca_, ea);
          test(base + 32 + lane, jb, sjb, Sb, cb, eb);
          decide(ja, sja, Sa, ca_, ea);
          if (base + 32 < total) decide(jb, sjb, Sb, cb, eb);
        }
      }
      for (int s = 0; s < nsp; ++s) {
        const int v = warp_sum(percnt[s]);
        if (lane == 0) b.seg_count[i * nsp + s] = v;
      }
      if (lane == 0) {
        b.slot_count[i] = cnt;
        atomicMax(b.max_count, cnt);
      }
    }
  }
}

cudaError_t sg_nbr_slots(const double* pos, const int* species, int n_atoms, int nsp, double rc,
                         int maxn, const NbrBuffers& b, cudaStream_t st) {
  cudaMemsetAsync(b.max_count, 0, sizeof(int), st);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // by bin pays when the bins alone fill the GPU: a single structure with a few bins per SM
  const bool by_atom = b.sweep == 2 || (b.sweep == 0 && (b.n_struct > 1 || b.n_bins < 8 * sms));
  if (n_atoms > 0 && by_atom) {
    const int threads = 128;
    const long long blocks = ((long long)n_atoms * 32 + threads - 1) / threads;
    fill_slots_kernel<<<(unsigned)blocks, threads, 0, st>>>(pos, species, n_atoms, nsp, rc, maxn, b,
                                                            b.binpos);
    ++sg_kernel_launches;
  } else if (n_atoms > 0 && b.n_bins > 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fill_slots_bins_kernel, NB_WARPS * 32, 0);
    const long long grid = std::min<long long>(b.n_bins, (long long)sms * std::max(1, per_sm));
    fill_slots_bins_kernel<<<(unsigned)grid, NB_WARPS * 32, 0, st>>>(pos, nsp, rc, maxn, b, b.binpos);
    ++sg_kernel_launches;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sg_exclusive_scan(b.seg_count, b.seg_offs, n_atoms * nsp, b.scan_tmp, st, b.run);
}

// Separation r = x_j + S.h - x_i of pair (i, j, S), exactly antisymmetric under
// (i, j, S) -> (j, i, -S): computed in the canonical orientation (j > i, or j = i with S
// lexicographically positive) and negated otherwise.
//   FP32 path: double-float sum of the split positions and the split shift, rounded once;
//   FP64 path: fixed-order FP64 operations without FMA.
template <typename T>
__device__ __forceinline__ Vec4<T> pair_vector(const double* __restrict__ pos, const NbrBuffers& b,
                                               int i, int j, int S1, int S2, int S3) {
  const StructGeom& g = b.geom[b.atom_struct[i]];
  const bool canon = (j > i) || (j == i && lex_positive(S1, S2, S3));
  if (b.img) {
    // list built from x - n h: with the positions as given the same pair has shift S - n_j + n_i
    const int4 ni = b.img[i], nj = b.img[j];
    S1 += ni.x - nj.x;
    S2 += ni.y - nj.y;
    S3 += ni.z - nj.z;
  }
  Vec4<T> v;
  if constexpr (sizeof(T) == 4) {
    const int pa = canon ? j : i, pb = canon ? i : j;
    const float4 ah4 = b.atom_hi[pa], al4 = b.atom_lo[pa];
    const float4 bh4 = b.atom_hi[pb], bl4 = b.atom_lo[pb];
    const float sg = canon ? 1.f : -1.f;
    const float ah[3] = {ah4.x, ah4.y, ah4.z}, al[3] = {al4.x, al4.y, al4.z};
    const float bh[3] = {bh4.x, bh4.y, bh4.z}, bl[3] = {bl4.x, bl4.y, bl4.z};
    float out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float sh, sl, th, tl, uh, ul;
      df_shift(g, sg * (float)S1, sg * (float)S2, sg * (float)S3, c, sh, sl);
      df_add(ah[c], al[c], sh, sl, th, tl);
      df_add(th, tl, -bh[c], -bl[c], uh, ul);
      out[c] = sg * __fadd_rn(uh, ul);
    }
    v.x = out[0];
    v.y = out[1];
    v.z = out[2];
    const float d2f = v.x * v.x + v.y * v.y + v.z * v.z;
    v.w = sqrtf(d2f);
    if (b.rc2_mask > 0.0) {
      // beyond r_cut (list built with a skin): decided like the list itself, FP32 away from
      // the cutoff (the double-float vector is within 2 ulp), the FP64 expression near it
      const float rc2f = (float)b.rc2_mask;
      bool beyond;
      if (fabsf(d2f - rc2f) > 16.f * 5.9604645e-8f * rc2f) {
        beyond = d2f >= rc2f;
      } else {
        double s[3], r[3], d2;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          s[c] = __dadd_rn(__dadd_rn(__dmul_rn((double)S1, g.h[c]), __dmul_rn((double)S2, g.h[3 + c])),
                           __dmul_rn((double)S3, g.h[6 + c]));
        exact_sep(pos, i, j, s, canon, r, d2);
        beyond = d2 >= b.rc2_mask;
      }
      if (beyond) v.w = -1.f;
    }
  } else {
    double s[3], r[3], d2;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      s[c] = __dadd_rn(__dadd_rn(__dmul_rn((double)S1, g.h[c]), __dmul_rn((double)S2, g.h[3 + c])),
                       __dmul_rn((double)S3, g.h[6 + c]));
    exact_sep(pos, i, j, s, canon, r, d2);
    v.x = r[0];
    v.y = r[1];
    v.z = r[2];
    v.w = (b.rc2_mask > 0.0 && d2 >= b.rc2_mask) ? -1.0 : sqrt(d2);
  }
  return v;
}

// Per atom (one warp): the slot keys, staged in shared memory with their neighbour
// species, are ranked within their species; each pair goes to its (centre, species)
// segment in key order with its j and separation vector.  Writes stay inside the segment
// (a segment emptied by the capacity guard receives nothing).
template <typename T>
__global__ void place_kernel(int n, int nsp, int maxn, const double* __restrict__ pos,
                             const int* __restrict__ species, NbrBuffers b, Vec4<T>* rout) {
  extern __shared__ __align__(16) unsigned long long sk[];
  if (b.run && *b.run == 0) return;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + wib;
  const int kstride = maxn + 2;  // one padding key, 16-byte aligned rows
  unsigned long long* keys = sk + (size_t)wib * kstride;
  unsigned char* spc = reinterpret_cast<unsigned char*>(sk + (size_t)(blockDim.x >> 5) * kstride) +
                       (size_t)wib * maxn;
  if (i >= n) return;
  const int cnt = min(b.slot_count[i], maxn);
  const unsigned long long* src = b.key_tmp + (size_t)i * maxn;
  for (int e = lane; e < cnt; e += 32) {
    const unsigned long long k = src[e];
    keys[e] = k;
    spc[e] = (unsigned char)(nsp > 1 ? species[(int)(k >> 24)] : 0);
  }
  __syncwarp();
  if ((cnt & 1) && lane == 0) keys[cnt] = ~0ull;  // pad to an even count for pairwise reads
  __syncwarp();
  const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(keys);
  const int n2 = (cnt + 1) >> 1;
  for (int e = lane; e < cnt; e += 32) {
    const unsigned long long k = keys[e];
    const int s = spc[e];
    int rank = 0;
    if (nsp == 1) {
      for (int o = 0; o < n2; ++o) {
        const ulonglong2 kk = k2[o];
        rank += (kk.x < k) + (kk.y < k);
      }
    } else {
      for (int o = 0; o < cnt; ++o) rank += (keys[o] < k) & (spc[o] == s);
    }
    const int at = b.seg_offs[i * nsp + s] + rank;
    if (at < b.seg_offs[i * nsp + s + 1]) {
      b.key[at] = k;
      const int j = (int)(k >> 24);
      b.pair_j[at] = j;
      const int s1 = (int)((k >> 16) & 255) - 128, s2 = (int)((k >> 8) & 255) - 128,
                s3 = (int)(k & 255) - 128;
      rout[at] = pair_vector<T>(pos, b, i, j, s1, s2, s3);
    }
  }
}

// reverse index: pair (i, j, S) -> position of (j, i, -S) in segment (j, species(i))
__global__ void rev_kernel(int n, int nsp, const int* __restrict__ species, NbrBuffers b) {
  if (b.run && *b.run == 0) return;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int si = species[i];
  const int beg = b.seg_offs[i * nsp], end = b.seg_offs[(i + 1) * nsp];
  for (int p = beg + lane; p < end; p += 32) {
    const unsigned long long k = b.key[p];
    const int j = (int)(k >> 24);
    const int s1 = (int)((k >> 16) & 255) - 128, s2 = (int)((k >> 8) & 255) - 128,
              s3 = (int)(k & 255) - 128;
    const unsigned long long want = pair_key(i, -s1, -s2, -s3);
    int lo = b.seg_offs[j * nsp + si], hi = b.seg_offs[j * nsp + si + 1] - 1, found = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const unsigned long long km = b.key[mid];
      if (km == want) { found = mid; break; }
      if (km < want) lo = mid + 1; else hi = mid - 1;
    }
    if (found < 0) atomicOr(b.err, SG_ERR_NO_REVERSE);
    b.rev[p] = found < 0 ? p : found;
  }
}

template <typename T>
cudaError_t sg_nbr_place(const double* pos, const int* species, int n_atoms, int nsp, int maxn,
                         const NbrBuffers& b, cudaStream_t st) {
  if (n_atoms == 0) return cudaSuccess;
  const int warps = 4;
  const size_t smem = (size_t)warps * ((maxn + 2) * 8 + maxn);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = sg_set_smem<place_kernel<T>>(smem);
  if (e != cudaSuccess) return e;
  place_kernel<T><<<(n_atoms + warps - 1) / warps, warps * 32, smem, st>>>(
      n_atoms, nsp, maxn, pos, species, b, reinterpret_cast<Vec4<T>*>(b.pair_r));
  const int threads = 128;
  const long long blocks = ((long long)n_atoms * 32 + threads - 1) / threads;
  rev_kernel<<<(unsigned)blocks, threads, 0, st>>>(n_atoms, nsp, species, b);
  sg_kernel_launches += 2;
  return cudaGetLastError();
}

template cudaError_t sg_nbr_place<float>(const double*, const int*, int, int, int, const NbrBuffers&,
                                         cudaStream_t);
template cudaError_t sg_nbr_place<double>(const double*, const int*, int, int, int, const NbrBuffers&,
                                          cudaStream_t);

// Pair-capacity guard of asynchronous calls: if the pair count (the last offset) exceeds
// the capacity, every segment is emptied and SG_ERR_PAIR_CAPACITY is raised, so that no
// later kernel indexes past the pair buffers.  One block: the decision is taken once.
__global__ void cap_guard_kernel(int* seg_offs, int nseg, long long cap, int* err, const int* run) {
  if (run && *run == 0) return;
  __shared__ int over;
  if (threadIdx.x == 0) {
    over = (long long)seg_offs[nseg] > cap || (*(volatile int*)err & SG_ERR_PAIR_CAPACITY) != 0;
    if (over) atomicOr(err, SG_ERR_PAIR_CAPACITY);
  }
  __syncthreads();
  if (!over) return;
  for (int k = threadIdx.x; k <= nseg; k += blockDim.x) seg_offs[k] = 0;
}

cudaError_t sg_nbr_cap_guard(int* seg_offs, int nseg, long long cap, int* err, cudaStream_t st,
                             const int* run) {
  cap_guard_kernel<<<1, 1024, 0, st>>>(seg_offs, nseg, cap, err, run);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Verlet skin
__global__ void skin_check_kernel(const double* __restrict__ pos, const double* __restrict__ ref, int n,
                                  double h2, int* rebuild) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dx = pos[3 * i] - ref[3 * i], dy = pos[3 * i + 1] - ref[3 * i + 1],
               dz = pos[3 * i + 2] - ref[3 * i + 2];
  if (dx * dx + dy * dy + dz * dz >= h2) *rebuild = 1;
}

cudaError_t sg_skin_check(const double* pos, const double* ref, int n, double half_skin,
                          int* rebuild, cudaStream_t st) {
  if (n > 0) {
    skin_check_kernel<<<(n + 255) / 256, 256, 0, st>>>(pos, ref, n, half_skin * half_skin, rebuild);
    ++sg_kernel_launches;
  }
  return cudaGetLastError();
}

// FP32 high / low words of the current positions (the double-float separations read them)
__global__ void split_positions_kernel(const double* __restrict__ pos, int n, NbrBuffers b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  const float xh = (float)x, yh = (float)y, zh = (float)z;
  b.atom_hi[i] = make_float4(xh, yh, zh, 0.f);
  b.atom_lo[i] = make_float4((float)(x - (double)xh), (float)(y - (double)yh), (float)(z - (double)zh), 0.f);
}

// Lists built with a skin, at every call: each pair's separation from its key and the
// current positions (|r| < 0 beyond r_cut), and the number of live pairs of each
// (centre, species) segment.  One warp per segment.
template <typename T>
__global__ void refresh_kernel(int nseg, int nsp, const double* __restrict__ pos, NbrBuffers b,
                               int* live_count, Vec4<T>* rout) {
  const int seg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (seg >= nseg) return;
  const int i = seg / nsp;
  const int beg = b.seg_offs[seg], end = b.seg_offs[seg + 1];
  int live = 0;
  for (int base = beg; base < end; base += 32) {
    const int p = base + lane;
    bool ok = false;
    if (p < end) {
      const unsigned long long k = b.key[p];
      const int j = (int)(k >> 24);
      const int s1 = (int)((k >> 16) & 255) - 128, s2 = (int)((k >> 8) & 255) - 128,
                s3 = (int)(k & 255) - 128;
      const Vec4<T> v = pair_vector<T>(pos, b, i, j, s1, s2, s3);
      rout[p] = v;
      ok = v.w >= T(0);
    }
    live += __popc(__ballot_sync(0xffffffffu, ok));
  }
  if (lane == 0) live_count[seg] = live;
}

// live pairs of each segment, in list (key) order: indices into the full list
template <typename T>
__global__ void live_fill_kernel(int nseg, NbrBuffers b, const int* __restrict__ live_offs,
                                 int* live_idx) {
  const int seg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (seg >= nseg) return;
  const int beg = b.seg_offs[seg], end = b.seg_offs[seg + 1];
  const Vec4<T>* pr = reinterpret_cast<const Vec4<T>*>(b.pair_r);
  int at = live_offs[seg];
  for (int base = beg; base < end; base += 32) {
    const int p = base + lane;
    const bool ok = p < end && pr[p].w >= T(0);
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (ok) live_idx[at + __popc(mask & ((1u << lane) - 1u))] = p;
    at += __popc(mask);
  }
}

template <typename T>
cudaError_t sg_nbr_refresh(const double* pos, int n_atoms, int nsp, const NbrBuffers& b,
                           int* live_count, int* live_offs, int* live_idx, cudaStream_t st) {
  if (n_atoms == 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    split_positions_kernel<<<(n_atoms + 255) / 256, 256, 0, st>>>(pos, n_atoms, b);
    ++sg_kernel_launches;
  }
  const int nseg = n_atoms * nsp;
  const int threads = 128;
  const long long blocks = ((long long)nseg * 32 + threads - 1) / threads;
  refresh_kernel<T><<<(unsigned)blocks, threads, 0, st>>>(nseg, nsp, pos, b, live_count,
                                                          reinterpret_cast<Vec4<T>*>(b.pair_r));
  ++sg_kernel_launches;
  cudaError_t e = sg_exclusive_scan(live_count, live_offs, nseg, b.scan_tmp, st);
  if (e != cudaSuccess) return e;
  live_fill_kernel<T><<<(unsigned)blocks, threads, 0, st>>>(nseg, b, live_offs, live_idx);
  ++sg_kernel_launches;
  return cudaGetLastError();
}
template cudaError_t sg_nbr_refresh<float>(const double*, int, int, const NbrBuffers&, int*, int*, int*,
                                           cudaStream_t);
template cudaError_t sg_nbr_refresh<double>(const double*, int, int, const NbrBuffers&, int*, int*, int*,
                                            cudaStream_t);

__global__ void skin_ref_kernel(const double* __restrict__ pos, double* ref, int n3, const int* rebuild) {
  if (rebuild && *rebuild == 0) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n3) ref[k] = pos[k];
}

cudaError_t sg_skin_ref_update(const double* pos, double* ref, int n, const int* rebuild,
                               cudaStream_t st) {
  if (n > 0) {
    skin_ref_kernel<<<(3 * n + 255) / 256, 256, 0, st>>>(pos, ref, 3 * n, rebuild);
    ++sg_kernel_launches;
  }
  return cudaGetLastError();
}
