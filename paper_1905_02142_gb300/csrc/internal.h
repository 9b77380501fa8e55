// Launch interfaces between the C-ABI layer (api.cu) and the kernel translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include "common.cuh"

// Raise kernel Kern's dynamic shared-memory limit, once per device and size: the attribute
// persists, and skipping repeated calls keeps a launch free of non-stream API calls (so
// that launches can be captured in a CUDA graph).
template <auto Kern>
inline cudaError_t sg_set_smem(size_t bytes) {
  static int done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if ((int)bytes <= done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[dev] = (int)bytes;
  return e;
}

// Kernels launched by this library since load (read around a call to count its launches).
extern std::atomic<long long> sg_kernel_launches;

// Compile-time capacity class of the pair kernels: (n_max, l_max) <= (NC, LC).
int sg_cap_class(int nmax, int lmax);            // 0..3 -> (6,6) (8,8) (10,10) (12,12)
int sg_cap_n(int cls);
int sg_cap_l(int cls);

// ---------------------------------------------------------------- basis_host.cpp
// W = S^-1/2 (row-major, FP64) from a binary128 computation; returns 0 or -1.
int sg_orthonormaliser_q(int nmax, double rc, double s0, double* W, double* cond);

// ---------------------------------------------------------------- tables.cu
struct TableInfo {
  int K;         // intervals
  int fp;        // floats per half-node (values, then h*derivatives): padded NC+LC+1
  double h;      // node spacing
  float inv_h;   // 1 / h (rounded to float)
};
// Builds, for r_k = k h (k = 0..K), b_n(r) in the orthonormal basis (n < nmax, padded to NC),
// 4 pi ilexp_l(z(r)) [x (2l+1) with eq08] (l <= lmax, padded to LC+1), and h * d/dr of each.
cudaError_t sg_build_table(const DevParams& p, const BasisConst<double>& W, int cls,
                           const TableInfo& ti, float* table, cudaStream_t st);
// FP16 operand scales of the tensor-core forward kernel (powers of two), from the table.
cudaError_t sg_fwd_mma_scales(const float* table, const TableInfo& ti, int ncp, int nmax, int lmax, float* sa,
                              float* sb);
// Central-atom constants: cen_n (orthonormal basis, for the table path) and cen_alpha.
cudaError_t sg_central_terms(const DevParams& p, const BasisConst<double>& W, double* out_n,
                             double* out_alpha, cudaStream_t st);

// ---------------------------------------------------------------- neighbours.cu
struct NbrBuffers {
  const StructGeom* geom;    // [S]
  const int* atom_struct;    // [N]
  int* atom_bin;             // [N] flattened bin index
  int4* atom_bin4;           // [N] bin coordinates within the structure's grid, and the index
  int* atom_slot;            // [N]
  int* bin_count;            // [nbins]
  int* bin_start;            // [nbins + 1]
  int* bin_atoms;            // [N]
  int* seg_count;            // [N*nsp]
  int* seg_offs;             // [N*nsp + 1]
  float4* binpos;            // [N] FP32 positions in bin order, .w = atom index
  float4* atom_hi;           // [N] FP32 positions, atom order
  float4* atom_lo;           // [N] their low words
  unsigned long long* key_tmp;  // [N][maxn] per-atom slots of kept pair keys (visit order)
  int* slot_count;           // [N] keys written per atom (may exceed maxn: overflow)
  int* max_count;            // [1] largest slot count
  unsigned long long* key;   // [cap]
  int* pair_j;               // [cap]
  void* pair_r;              // [cap] Vec4<T>
  int* rev;                  // [cap]
  int* scan_tmp;             // scan scratch
  int* err;                  // device error word
  const int4* img;           // if set: cell image n_i of each atom at the last build (the list
                             // was built from x - n_i h); separations then use the positions
                             // as given with the shift S - n_j + n_i
  const int* run;            // if set and *run == 0, the list-building kernels return at once
                             // (neighbour-list reuse decided on the device)
  double rc2_mask;           // > 0: pairs with |r|^2 >= rc2_mask get |r| = -1 (beyond r_cut
                             // in a list built with a skin); 0: no masking
  int n_struct, n_bins;      // structures and bins of the batch
  int sweep;                 // candidate sweep: 1 one block per bin, 2 one warp per atom, 0 chosen
                             // from the batch (per bin for one structure of many bins)
};
size_t sg_scan_tmp_ints(int n);
cudaError_t sg_exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t st,
                              const int* run = nullptr);
// positions mapped into their cells for the list build: pos_w = x - n h with n = floor of the
// fractional coordinates (n = 0, pos_w = x exactly, for atoms inside up to 1e-9), img = n
cudaError_t sg_nbr_wrap(const double* pos, int n_atoms, const NbrBuffers& b, double* pos_w,
                        int4* img, cudaStream_t st);
cudaError_t sg_nbr_bin(const double* pos, const int* species, int n_atoms, int n_bins, const NbrBuffers& b,
                       cudaStream_t st);
// one sweep over the candidates: per-atom slot arrays of keys (capacity maxn), counts per
// (atom, species) segment, their exclusive scan into seg_offs, and the largest count
cudaError_t sg_nbr_slots(const double* pos, const int* species, int n_atoms, int nsp, double rc,
                         int maxn, const NbrBuffers& b, cudaStream_t st);
// asynchronous calls: empty all segments and flag SG_ERR_PAIR_CAPACITY if seg_offs[nseg] > cap
// or a slot array overflowed
cudaError_t sg_nbr_cap_guard(int* seg_offs, int nseg, long long cap, int* err, cudaStream_t st,
                             const int* run = nullptr);
// Verlet skin: rebuild[0] |= 1 if an atom moved by skin/2 or more since the positions `ref`
// of the last build; refresh recomputes every pair's separation from its key and the current
// positions (|r| < 0 beyond r_cut) and lists the live pairs of each segment (live_offs
// [N*nsp + 1], live_idx: indices into the full list); ref_update copies pos to ref if *rebuild
cudaError_t sg_skin_check(const double* pos, const double* ref, int n, double half_skin,
                          int* rebuild, cudaStream_t st);
template <typename T>
cudaError_t sg_nbr_refresh(const double* pos, int n_atoms, int nsp, const NbrBuffers& b,
                           int* live_count, int* live_offs, int* live_idx, cudaStream_t st);
cudaError_t sg_skin_ref_update(const double* pos, double* ref, int n, const int* rebuild,
                               cudaStream_t st);
// keys ranked into their segments with j and the separation vectors, then the reverse index
template <typename T>
cudaError_t sg_nbr_place(const double* pos, const int* species, int n_atoms, int nsp, int maxn,
                         const NbrBuffers& b, cudaStream_t st);

// ---------------------------------------------------------------- pair_fwd.cu
template <typename T> struct FwdArgs {
  int n_atoms, nsp, nmax, lmax;
  const int* species;
  const int* seg_offs;      // segment offsets of the pairs to use
  const int* pair_idx;      // if set: index into pair_r of each of those pairs (live pairs)
  const Vec4<T>* pair_r;
  const float* table;     // table path
  TableInfo ti;
  DevParams p;            // recursion path
  YlmCoef<T> yc;
  BasisConst<T> bc;       // W (recursion path) and central terms (both)
  T* c;                   // [N][nsp*nmax][L]
  int* err;               // device error word (SG_ERR_TIMEOUT if a table copy never lands)
  float mma_sa, mma_sb;   // tensor-core forward: powers of two scaling a_lm and b_n into FP16 range
};
template <typename T> cudaError_t sg_pair_forward(const FwdArgs<T>& a, int cls, bool table,
                                                  cudaStream_t st);
// Mixed path: the same coefficients with the neighbour contraction on tensor cores
// (pair_fwd_mma.cu); needs mma_sa, mma_sb (sg_fwd_mma_scales).
bool sg_pair_forward_mma_supported(int cls);
cudaError_t sg_pair_forward_mma(const FwdArgs<float>& a, int cls, cudaStream_t st);

// ---------------------------------------------------------------- powspec.cu
// The mixed path's GAP operand of each atom, written by the power-spectrum kernel when a16
// is set (the same values as sg_gap_tc_prepare; FP32 descriptors only).
struct GapOperand {
  __half* a16;        // [N][terms * dp]
  float* nrm;         // [N] |q - qbar|
  float* uq;          // [N] qbar.(q - qbar)
  const float* qbar;  // [dp]
  int dp, terms;
};
template <typename T>
cudaError_t sg_power_spectrum(const T* c, int n_atoms, int nch, int lmax, int lc, T* q, T* pnorm,
                              cudaStream_t st, const GapOperand& op = GapOperand{});  // lc: class bound on l_max

// ---------------------------------------------------------------- gap_simt.cu
// eps_part[i][t] = sum over sparse tile t of alpha_s S_is^zeta,
// kp[i][s] = zeta alpha_s S_is^(zeta-1)   (kp may be NULL: energy only)
template <typename T>
cudaError_t sg_gap_forward_simt(const T* q, const T* qs, const T* alpha, int n, int m, int d,
                                double zeta, T* eps_part, int n_tiles, T* kp, cudaStream_t st);
int sg_gap_tiles(int m);
// g[i][k] = sum_s kp[i][s] qs[s][k]
template <typename T>
cudaError_t sg_gap_backward_simt(const T* kp, const T* qs, int n, int m, int d, T* g,
                                 cudaStream_t st);

// ---------------------------------------------------------------- gap_tc.cu
// Sparse-set side of the tensor-core GAP kernels (built by soapgap_set_model).
struct GapTcModel {
  int d, dp, mp, izeta;   // D, D padded to 64, M padded to 256, integer zeta (0: not integer)
  float c0, zeta, kappa;  // qbar.qbar, zeta, backward scale
  const __half* B;        // [mp][3 dp]  unit centred sparse rows as [hi | lo | hi]
  const __half* BT;       // [dp][mp]    the same rows transposed, hi only
  const float4* col;      // [mp]: (qbar.qbar + qbar.(q_s - qbar), |q_s - qbar|, alpha_s,
                          //        zeta alpha_s |q_s - qbar| / kappa), zero beyond M
  const float* qbar;      // [dp]
  // force rows of the fitting matrices: A = [kd (q_s - qbar) | kd | kd | 0 ...] per sparse
  // row, so that A . [J' | hi(qbar.J') | lo(qbar.J')] = kd q_s . J' (see design.cu)
  int dpd;                // D + 2 padded to 64
  float kd;               // power of two: max |kd (q_s - qbar)| in [1, 2)
  const __half* Ad;       // [mp][dpd]
  int terms;              // FP16 products of the energy: 1 (hi.hi) or 3 (hi.hi + hi.lo + lo.hi)
  int fwd_cfg, bwd_cfg;   // tile configurations of the forward and backward products
};
#define SG_GAP_FWD_CFGS 3
#define SG_GAP_BWD_CFGS 5
// partial-sum slots per atom row of the forward product with configuration fwd_cfg, and
// the most any configuration needs
int sg_gap_tc_tiles(int mp, int fwd_cfg);
int sg_gap_tc_tiles_max(int mp);
// A rows of the atoms: terms = 1 gives [hi] (row stride dp; the energy and its gradient),
// terms = 3 the split [hi | hi | lo] (row stride 3 dp; kernel rows of the fitting matrices)
cudaError_t sg_gap_tc_prepare(const float* q, int n, int d, int dp, const float* qbar, __half* A,
                              float* nrm, float* uq, int terms, cudaStream_t st);
// energy epilogue over `terms` FP16 products (1 or 3): A from sg_gap_tc_prepare with the same terms
cudaError_t sg_gap_tc_forward(const GapTcModel& md, int terms, const __half* A, const float* nrm,
                              const float* uq, int n, float* eps_part, float* r_part, __half* kp, int* err,
                              cudaStream_t st);
cudaError_t sg_gap_tc_backward(const GapTcModel& md, const __half* kp, const float* r_part, int n,
                               float* g, int* err, cudaStream_t st);
cudaError_t sg_tc_gemm_store(const __half* A, int m, const __half* B, int n, int k, float* C, int* err,
                             cudaStream_t st);

// ---------------------------------------------------------------- pair_adj.cu
template <typename T> struct AdjArgs {
  int n_atoms, nsp, nmax, lmax, dim;
  long long n_pairs;
  int warps;                // warps per block of the tensor-core adjoint (0: from n_pairs)
  const int* species;
  const int* atom_struct;
  const double* struct_w;   // [S] dE/dE_struct
  const int* seg_offs;      // segment offsets of the pairs to use
  const int* pair_idx;      // if set: index into pair_r / dedr of each of those pairs
  const int* list_offs;     // segment offsets of the full list (prefetch ranges)
  const Vec4<T>* pair_r;
  const float* table;
  TableInfo ti;
  DevParams p;
  YlmCoef<T> yc;
  BasisConst<T> bc;
  const T* c;               // [N][nch][L]
  const T* q;               // [N][D]
  const T* pnorm;           // [N]
  const T* g;               // [N][D] dE/dq (before the structure weight)
  Vec4<T>* dedr;            // [P] dE/dr_ij
  T* vir_atom;              // [N][9]
  int* err;                 // device error word (SG_ERR_*)
  unsigned char* gimg;      // tcgen05 variant: per atom, the FP16 operand image of dE/dc
  int* gexp;                //   (sg_adj_tc_image_bytes bytes) and its power-of-two exponent
};
template <typename T> cudaError_t sg_pair_adjoint(const AdjArgs<T>& a, int cls, bool table,
                                                  cudaStream_t st);
// mixed-precision (table) adjoint with the per-atom contraction on tensor cores
cudaError_t sg_pair_adjoint_mma(const AdjArgs<float>& a, int cls, cudaStream_t st);
// the tcgen05 variant (pair_adj_tc.cu), selected by a.warps == SG_ADJ_TCGEN05; only for
// exact basis sizes of the class (n_max = l_max = 6 + 2 cls)
#define SG_ADJ_TCGEN05 5
bool sg_pair_adjoint_tc_supported(const AdjArgs<float>& a, int cls);
cudaError_t sg_pair_adjoint_tc(const AdjArgs<float>& a, int cls, cudaStream_t st);
// bytes of one atom's operand image of the tcgen05 variant (a.gimg holds n_atoms of them)
size_t sg_adj_tc_image_bytes(int cls, int nsp);
// 32-pair batches of a typical atom (sum over its neighbour-species segments)
int sg_adj_batches_per_atom(long long n_pairs, int n_atoms, int nsp);

// ---------------------------------------------------------------- design.cu
// Columns of the force rows of the fitting matrices: J_ij = dp_i/dr_ij (3 per pair, stored
// at the slot of the reverse pair in the target's range) and -sum_j J_ij (3 self columns per
// atom, after the target's pairs): column range of atom k = [3 (o_k + k), 3 (o_(k+1) + k + 1)).
template <typename T> struct JacArgs {
  int n_atoms, nsp, nmax, lmax, dim;
  int ld;                   // row length of a stored column (D padded to 64 for FP16, D for FP64)
  const int* seg_offs;      // [N*nsp + 1] the full list
  const int* rev;           // [P]
  const int* pair_j;        // [P]
  const Vec4<T>* pair_r;    // [P] (|r| < 0: masked pair, zero columns)
  const float* table;       // table path
  TableInfo ti;
  DevParams p;              // recursion path
  YlmCoef<T> yc;
  BasisConst<T> bc;
  const T* c;               // [N][nch][L]
  const T* q;               // [N][D]
  const float* qbar;        // [D] sparse-set mean (table path)
  void* J;                  // [ncols][ld]: table path __half [2^e J' | hi, lo of 2^e qbar.J' | 0],
                            // J' = J - q_owner (q_owner . J), one e per column triple; FP64 path J
  int2* col_at;             // [ncols] (owner atom, target atom)
  Vec4<T>* col_v;           // [ncols] (qbar . J, q_owner . J, 2^-e, 0), unprojected J
};
template <typename T> cudaError_t sg_design_jacobian(const JacArgs<T>& a, int cls, bool table,
                                                     cudaStream_t st);
// FP64 path: k[i][s] = (q_i.q_s)^zeta and, if wv, wv[i][s] = (w, w S) with
// w = zeta S^(zeta-1) / |p_i| (row stride ldw)
cudaError_t sg_kernel_rows_f64(const double* q, int n, const double* qs, int m, int d, double zeta,
                               const double* pnorm, double* k, double2* wv, int ldw, cudaStream_t st);
// FP64 path: dk[target][a][s] += w_os (q_s . J_col) - (w S)_os (q_o . J_col) for every column
cudaError_t sg_design_grad_f64(const double* qs, int m, int d, const double* J, long long ncols,
                               const int2* col_at, const Vec4<double>* col_v, const double2* wv, int ldw,
                               double* dk, cudaStream_t st);
// out[t][s] += sum over the atoms i of structure t of k[i][s]  (out zeroed by the caller)
template <typename T>
cudaError_t sg_struct_rows(const T* k, int n, int m, const int* atom_struct, double* out, cudaStream_t st);
// mixed path (gap_tc.cu): kernel rows from the prepared FP16 split operands, and the force
// rows from the FP16 columns on tensor cores
cudaError_t sg_tc_kernel_rows(const GapTcModel& md, const __half* A, const float* nrm, const float* uq, int n,
                              int m, const float* pnorm, float* k, float2* wv, int* err, cudaStream_t st);
cudaError_t sg_tc_design_grad(const GapTcModel& md, int m, const __half* J, long long ncols, const int2* col_at,
                              const float4* col_v, const float2* wv, float* dk, int* err, cudaStream_t st);

// ---------------------------------------------------------------- forces.cu
// chunks per structure of the two-level per-structure sums (part: [S][chunks][10] doubles)
int sg_finish_chunks(int max_struct_atoms);
// velocity-Verlet half step (kick; with drift also the position update)
cudaError_t sg_verlet(int n, double* pos, double* vel, const double* forces, const double* inv_mass,
                      double dt, bool drift, cudaStream_t st);
template <typename T>
cudaError_t sg_finish(int n_atoms, int n_struct, int nsp, const int64_t* atom_offs_dev,
                      const int* seg_offs, const int* pair_idx, const int* rev, const Vec4<T>* dedr,
                      const T* eps_part, int n_tiles, const T* vir_atom, T* e_atom,
                      double* e_struct, double* forces, double* virial, bool sign_force,
                      int chunks, double* part, cudaStream_t st);
