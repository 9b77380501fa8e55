// C ABI of the library (declared in include/soapgap.h): argument checks, FP64 set-up of
// the radial basis on the host, the device workspace, and the launch sequence of one
// evaluation.  No exception crosses the ABI; every failure returns a negative code and
// leaves a message in the handle.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/soapgap.h"
#include "internal.h"
#include "soapmath.cuh"

// --------------------------------------------------------------------- helpers
std::atomic<long long> sg_kernel_launches{0};

int sg_cap_class(int nmax, int lmax) {
  int m = nmax > lmax ? nmax : lmax;
  return m <= 6 ? 0 : (m <= 8 ? 1 : (m <= 10 ? 2 : 3));
}
int sg_cap_n(int cls) { return 6 + 2 * cls; }
int sg_cap_l(int cls) { return 6 + 2 * cls; }

namespace {

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

cudaError_t ensure(Buf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 4 + 256;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) return e;
  b.cap = want;
  return cudaSuccess;
}

template <typename T> YlmCoef<T> ylm_coefficients() {
  YlmCoef<T> y;
  std::memset(&y, 0, sizeof(y));
  for (int m = 0; m <= SG_MAX_LMAX; ++m) {
    double prod = 1.0;
    for (int k = 1; k <= m; ++k) prod *= (2.0 * k - 1.0) / (2.0 * k);
    double seed = std::sqrt((2.0 * m + 1.0) / (4.0 * M_PI) * prod);
    if (m > 0) seed *= std::sqrt(2.0);
    y.seed[m] = (T)seed;
    y.s1[m] = (T)std::sqrt(2.0 * m + 3.0);
    for (int l = 0; l <= SG_MAX_LMAX; ++l) {
      if (l >= m + 2) {
        double l2 = (double)l * l, m2 = (double)m * m;
        y.a[l][m] = (T)std::sqrt((4.0 * l2 - 1.0) / (l2 - m2));
        y.b[l][m] = (T)std::sqrt((2.0 * l + 1.0) * ((l - 1.0) * (l - 1.0) - m2) /
                                 ((2.0 * l - 3.0) * (l2 - m2)));
      }
      if (l >= m) {
        double d = std::sqrt((double)(l - m) * (l + m + 1));
        if (m == 0) d /= std::sqrt(2.0);
        y.d[l][m] = (T)d;
      }
    }
  }
  return y;
}

}  // namespace

struct soapgap_handle {
  soapgap_params prm;
  DevParams dp;
  int cls = 0, NC = 0, LC = 0;
  int D = 0, nch = 0, L = 0;
  bool mixed = false;
  BasisConst<double> bc64;   // W and cen_alpha (recursion path)
  BasisConst<float> bc32;    // cen_n (table path)
  YlmCoef<float> yc32;
  YlmCoef<double> yc64;
  TableInfo ti{}, ti_adj{};
  Buf table, table_adj;      // radial tables: descriptors (and fitting rows), adjoint
  float fwd_sa = 0.f, fwd_sb = 0.f;  // FP16 operand scales of the tensor-core forward
  // model
  int M = 0;
  double zeta = 0;
  Buf qs, alpha;
  bool has_model = false;
  // tensor-core GAP operands of the sparse set (mixed path)
  Buf tc_B, tc_BT, tc_cols, tc_qbar, tc_Ad;
  GapTcModel tcm{};
  Buf A16, nrm, uq, r_part, kp16;
  int gap_terms_forced = 0;      // 0: chosen per model from the probe below; 1 or 3: forced
  double gap_probe_err = -1.0;   // one-product error of the energy on the sparse rows
  // workspace
  Buf geom, atom_offs, atom_struct, atom_bin, atom_bin4, atom_slot, bin_count, bin_start, bin_atoms, binpos,
      atom_hi, atom_lo;
  Buf seg_count, seg_offs, scan_tmp, key_tmp, key, pair_j, pair_r, rev, dedr, slot_count, max_count;
  Buf adj_img, adj_exp;      // tcgen05 adjoint: per-atom G operand images and their exponents
  // Verlet skin: the list holds pairs within r_cut + skin and is reused while no atom has
  // moved by skin/2 since the positions pos_ref of its build
  double skin = 0.0;
  Buf pos_ref, skin_flag, live_count, live_offs, live_idx;
  Buf pos_w, img;           // positions mapped into their cells at the last build, and n_i
  bool ref_valid = false;
  int ref_atoms = -1, ref_struct = -1;
  std::vector<double> ref_cell;
  int last_rebuild = -1;    // 1 / 0 for synchronous calls, -1 when decided on the device
  bool list_ok = false;     // the pair list (seg_offs, key) is complete, with last_pairs pairs
  int list_atoms = 0;       // ... over this many atoms
  int slot_maxn = 0;        // slot capacity per atom of the last synchronous neighbour search
  int cur_maxn = 0;         // slot capacity used by the current call
  int slot_maxn_est = 0;    // estimate for the current batch (from its densities)
  Buf c, q, pnorm, e_atom, eps_part, kp, g, vir_atom, struct_w, err, cen_tmp, finish_part;
  int finish_chunks = 1;
  Buf host_in_pos, host_in_species, host_q, host_pnorm, host_e_atom, host_e_struct, host_forces,
      host_virial;
  int* h_err = nullptr;           // pinned
  int* h_count = nullptr;         // pinned
  int* h_err_async = nullptr;     // pinned: device error word of the last asynchronous call
  int64_t* h_offs = nullptr;      // pinned staging of atom_offs (read by captured copies)
  size_t h_offs_cap = 0;
  bool async_call = false;        // current call must not allocate or synchronise
  // tile plan per problem class (soapgap_autotune / soapgap_set_plan): adjoint warps per
  // block (0: by pairs per atom) and the configurations of the two GAP products
  struct TilePlan { int adj_warps = 0, gap_fwd = 0, gap_bwd = 0, nbr_sweep = 0, pair_fwd = 0; };
  std::map<long long, TilePlan> plans;
  StructGeom* h_geom = nullptr;   // pinned staging
  size_t h_geom_cap = 0;
  double* h_w = nullptr;
  size_t h_w_cap = 0;
  std::string msg;
  int64_t last_pairs = 0;
  int fw_atoms = -1, fw_struct = -1;
  bool have_forward = false;
  int n_bins = 0;
  // stage timing: events recorded around the stages of one call on the caller's stream
  cudaEvent_t ev[10] = {};
  bool ev_made = false, timed = false;
  bool stage_ran[SOAPGAP_N_STAGES] = {};
  long long launches = 0;
  // fitting-matrix rows (soapgap_design): kernel rows when not returned, force-row weights,
  // Jacobian columns and their (owner, target) and (qbar.J, q.J, 1/scale) records
  Buf dk_k, dk_wv, dk_J, dk_at, dk_v;
  cudaEvent_t dev_ev[SOAPGAP_N_DESIGN_STAGES + 1] = {};
  bool dev_made = false, dev_timed = false;
  bool dstage_ran[SOAPGAP_N_DESIGN_STAGES] = {};
};

// event slots: 0/1 neighbour search before the size read-back, 2/3 the fill after it,
// then 3..9 bound the stages pair_forward .. finish
enum { EV_NB0 = 0, EV_NB1, EV_FILL0, EV_FWD0, EV_PS0, EV_GF0, EV_GB0, EV_ADJ0, EV_FIN0, EV_END };

static void mark(soapgap_handle* h, int slot, cudaStream_t st) {
  if (h->timed) cudaEventRecord(h->ev[slot], st);
}

static int fail(soapgap_handle* h, int code, const std::string& m) {
  if (h) h->msg = m;
  return code;
}

#define CK(h, x)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (x);                                                               \
    if (e_ != cudaSuccess)                                                              \
      return fail((h), SOAPGAP_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// workspace growth; an asynchronous call (SOAPGAP_ASYNC) may only use what earlier calls
// allocated
#define ENS(h, buf, bytes)                                                                  \
  do {                                                                                      \
    const size_t b_ = (bytes);                                                              \
    if ((h)->async_call) {                                                                  \
      if (!(buf).p || (buf).cap < b_)                                                       \
        return fail((h), SOAPGAP_E_STATE,                                                   \
                    "workspace too small for an asynchronous call (" #buf                   \
                    "): make one synchronous call with the same batch first");             \
    } else {                                                                                \
      CK((h), ensure((buf), b_));                                                           \
    }                                                                                       \
  } while (0)

static int check_params(const soapgap_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return SOAPGAP_E_INVALID_ARG; }
  if (!(p->r_cut > 0) || !std::isfinite(p->r_cut)) { why = "r_cut must be > 0"; return SOAPGAP_E_INVALID_ARG; }
  if (!(p->r_soft > 0) || p->r_soft > p->r_cut) { why = "need 0 < r_soft <= r_cut"; return SOAPGAP_E_INVALID_ARG; }
  if (!(p->sigma_r0 > 0) || !(p->sigma_p0 > 0)) { why = "atom sigmas must be > 0"; return SOAPGAP_E_INVALID_ARG; }
  if (!(p->alpha_r >= 0) || !(p->alpha_p >= 0) || !(p->amp_a >= 0)) { why = "alpha_r, alpha_p, amp_a must be >= 0"; return SOAPGAP_E_INVALID_ARG; }
  if (p->r_soft < p->r_cut && !(p->n_f > 0)) { why = "n_f must be > 0"; return SOAPGAP_E_INVALID_ARG; }
  if (!std::isfinite(p->central_weight)) { why = "central_weight must be finite"; return SOAPGAP_E_INVALID_ARG; }
  if (p->precision != SOAPGAP_FP64 && p->precision != SOAPGAP_MIXED) { why = "precision must be FP64 or MIXED"; return SOAPGAP_E_INVALID_ARG; }
  if (p->eq08_weight != 0 && p->eq08_weight != 1) { why = "eq08_weight must be 0 or 1"; return SOAPGAP_E_INVALID_ARG; }
  if (p->n_max < 2 || p->n_max > SOAPGAP_MAX_NMAX) { why = "n_max must be in [2, 12] (the basis degenerates beyond 12)"; return SOAPGAP_E_UNSUPPORTED; }
  if (p->l_max < 0 || p->l_max > SOAPGAP_MAX_LMAX) { why = "l_max must be in [0, 12]"; return SOAPGAP_E_UNSUPPORTED; }
  if (p->n_species < 1 || p->n_species > SOAPGAP_MAX_SPECIES) { why = "n_species must be in [1, 8]"; return SOAPGAP_E_UNSUPPORTED; }
  return SOAPGAP_OK;
}

extern "C" int soapgap_create(const soapgap_params* params, soapgap_handle** out) {
  if (!out) return SOAPGAP_E_INVALID_ARG;
  *out = nullptr;
  std::string why;
  int rc = check_params(params, why);
  if (rc != SOAPGAP_OK) {
    std::fprintf(stderr, "soapgap_create: %s\n", why.c_str());
    return rc;
  }
  soapgap_handle* h = new (std::nothrow) soapgap_handle();
  if (!h) return SOAPGAP_E_CUDA;
  h->prm = *params;
  const soapgap_params& p = *params;
  h->dp = DevParams{p.r_cut, p.r_soft, p.sigma_r0, p.sigma_p0, p.alpha_r, p.alpha_p, p.amp_a,
                    p.n_f, p.central_weight, p.n_max, p.l_max, p.n_species, p.eq08_weight};
  h->cls = sg_cap_class(p.n_max, p.l_max);
  h->NC = sg_cap_n(h->cls);
  h->LC = sg_cap_l(h->cls);
  h->nch = p.n_species * p.n_max;
  h->L = (p.l_max + 1) * (p.l_max + 1);
  h->D = h->nch * (h->nch + 1) / 2 * (p.l_max + 1);
  h->mixed = p.precision == SOAPGAP_MIXED;
  // W = S^-1/2: built in binary128 on the host, rounded to FP64 (Sec. III.A)
  double Wd[SG_MAX_NMAX * SG_MAX_NMAX], cond = 0;
  if (sg_orthonormaliser_q(p.n_max, p.r_cut, p.sigma_r0, Wd, &cond) != 0) {
    delete h;
    std::fprintf(stderr, "soapgap_create: overlap matrix is not positive definite\n");
    return SOAPGAP_E_UNSUPPORTED;
  }
  std::memset(&h->bc64, 0, sizeof(h->bc64));
  std::memset(&h->bc32, 0, sizeof(h->bc32));
  for (int a = 0; a < p.n_max; ++a)
    for (int b = 0; b < p.n_max; ++b) {
      h->bc64.W[a][b] = Wd[a * p.n_max + b];
    }
  h->yc32 = ylm_coefficients<float>();
  h->yc64 = ylm_coefficients<double>();
  // central-atom constants (and the radial table for the mixed path)
  cudaError_t e = ensure(h->cen_tmp, 2 * SG_MAX_NMAX * sizeof(double));
  if (e == cudaSuccess) e = sg_central_terms(h->dp, h->bc64, (double*)h->cen_tmp.p,
                                             (double*)h->cen_tmp.p + SG_MAX_NMAX, 0);
  double cen[2 * SG_MAX_NMAX];
  if (e == cudaSuccess) e = cudaMemcpy(cen, h->cen_tmp.p, sizeof(cen), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    for (int n = 0; n < p.n_max; ++n) {
      h->bc32.cen[n] = (float)cen[n];
      h->bc64.cen[n] = cen[SG_MAX_NMAX + n];
    }
    if (h->mixed) {
      double smin = std::min(p.sigma_r0, p.sigma_p0);
      double ht = std::min(0.02, smin / 25.0);
      h->ti.K = (int)std::ceil(p.r_cut / ht);
      h->ti.h = p.r_cut / h->ti.K;
      h->ti.inv_h = (float)(1.0 / h->ti.h);
      h->ti.fp = (h->NC + 3) / 4 * 4 + (h->LC + 1 + 3) / 4 * 4;  // TableDims<NC, LC>::FP
      e = ensure(h->table, (size_t)(h->ti.K + 1) * 2 * h->ti.fp * sizeof(float));
      if (e == cudaSuccess) e = sg_build_table(h->dp, h->bc64, h->cls, h->ti, (float*)h->table.p, 0);
      // The adjoint only feeds forces and virial (bar 1e-3 RMS), and reads the table of every
      // pair together with its derivative: it takes nodes four times as far apart (a quarter
      // of the table, which then stays in L1), with interpolation errors of about 6e-5 on the
      // values and 6e-5 RMS (9e-4 at most) on the derivatives, relative to each function's
      // scale, against 2.4e-7 and 9e-7 RMS for the descriptor table.
      double ha = std::min(0.08, smin / 6.25);
      h->ti_adj = h->ti;
      h->ti_adj.K = (int)std::ceil(p.r_cut / ha);
      h->ti_adj.h = p.r_cut / h->ti_adj.K;
      h->ti_adj.inv_h = (float)(1.0 / h->ti_adj.h);
      if (e == cudaSuccess) e = ensure(h->table_adj, (size_t)(h->ti_adj.K + 1) * 2 * h->ti_adj.fp * sizeof(float));
      if (e == cudaSuccess) e = sg_build_table(h->dp, h->bc64, h->cls, h->ti_adj, (float*)h->table_adj.p, 0);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e == cudaSuccess)
        e = sg_fwd_mma_scales((const float*)h->table.p, h->ti, (h->NC + 3) / 4 * 4, p.n_max, p.l_max, &h->fwd_sa,
                              &h->fwd_sb);
    }
  }
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_count, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_err_async, sizeof(int));
  if (e == cudaSuccess) *h->h_err_async = 0;
  if (e == cudaSuccess) e = ensure(h->err, sizeof(int));
  if (e != cudaSuccess) {
    std::fprintf(stderr, "soapgap_create: CUDA error: %s\n", cudaGetErrorString(e));
    soapgap_destroy(h);
    return SOAPGAP_E_CUDA;
  }
  *out = h;
  return SOAPGAP_OK;
}

extern "C" int soapgap_orthonormaliser(int32_t n_max, double r_cut, double sigma_r0, double* W) {
  if (!W || !(r_cut > 0) || !(sigma_r0 > 0)) return SOAPGAP_E_INVALID_ARG;
  if (n_max < 2 || n_max > SOAPGAP_MAX_NMAX) return SOAPGAP_E_UNSUPPORTED;
  double cond = 0;
  return sg_orthonormaliser_q(n_max, r_cut, sigma_r0, W, &cond) == 0 ? SOAPGAP_OK : SOAPGAP_E_UNSUPPORTED;
}

extern "C" int soapgap_descriptor_dim(const soapgap_handle* h, int32_t* dim) {
  if (!h || !dim) return SOAPGAP_E_INVALID_ARG;
  *dim = h->D;
  return SOAPGAP_OK;
}

static std::string device_error_text(int code);
static soapgap_handle::TilePlan plan_for(const soapgap_handle* h, int n_atoms);

extern "C" int soapgap_set_model(soapgap_handle* h, const double* q_sparse, const double* alpha,
                                 int32_t m, double zeta) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  if (!q_sparse || !alpha || m < 1) return fail(h, SOAPGAP_E_INVALID_ARG, "set_model: need q_sparse, alpha and m >= 1");
  if (!(zeta > 0) || !std::isfinite(zeta)) return fail(h, SOAPGAP_E_INVALID_ARG, "set_model: zeta must be > 0");
  const size_t nq = (size_t)m * h->D;
  for (size_t i = 0; i < nq; ++i)
    if (!std::isfinite(q_sparse[i])) return fail(h, SOAPGAP_E_INVALID_ARG, "set_model: q_sparse is not finite");
  for (int i = 0; i < m; ++i)
    if (!std::isfinite(alpha[i])) return fail(h, SOAPGAP_E_INVALID_ARG, "set_model: alpha is not finite");
  // The buffers below may be reallocated: until they all hold the new model the handle has
  // none, so a failure part-way leaves no stale device pointer in use.
  h->has_model = false;
  h->have_forward = false;
  h->M = 0;
  h->tcm = GapTcModel{};
  h->gap_probe_err = -1.0;
  const size_t es = h->mixed ? sizeof(float) : sizeof(double);
  CK(h, ensure(h->qs, nq * es));
  CK(h, ensure(h->alpha, (size_t)m * es));
  if (h->mixed) {
    std::vector<float> a(nq), b(m);
    for (size_t i = 0; i < nq; ++i) a[i] = (float)q_sparse[i];
    for (int i = 0; i < m; ++i) b[i] = (float)alpha[i];
    CK(h, cudaMemcpy(h->qs.p, a.data(), nq * es, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->alpha.p, b.data(), (size_t)m * es, cudaMemcpyHostToDevice));
    // Tensor-core operands (FP64 on the host, then rounded): centre on the sparse mean,
    // scale each centred row to unit norm, split it into FP16 hi + lo.
    const int D = h->D, dp = (D + 63) / 64 * 64, mp = (m + 255) / 256 * 256;
    std::vector<double> qbar(D, 0.0);
    for (int s = 0; s < m; ++s)
      for (int k = 0; k < D; ++k) qbar[k] += q_sparse[(size_t)s * D + k];
    for (int k = 0; k < D; ++k) qbar[k] /= m;
    double c0 = 0.0;
    for (int k = 0; k < D; ++k) c0 += qbar[k] * qbar[k];
    std::vector<__half> B((size_t)mp * 3 * dp, __float2half_rn(0.f)), BT((size_t)dp * mp, __float2half_rn(0.f));
    std::vector<float> cols(4 * (size_t)mp, 0.f), qb(dp, 0.f);  // float4 per column
    double kappa = 0.0;
    std::vector<double> nrm(m);
    std::vector<double> u(D);
    for (int s = 0; s < m; ++s) {
      double ss = 0.0, t = 0.0;
      for (int k = 0; k < D; ++k) {
        const double x = q_sparse[(size_t)s * D + k] - qbar[k];
        ss += x * x;
        t += x * qbar[k];
      }
      nrm[s] = std::sqrt(ss);
      cols[4 * (size_t)s] = (float)(c0 + t);
      cols[4 * (size_t)s + 1] = (float)nrm[s];
      cols[4 * (size_t)s + 2] = (float)alpha[s];
      kappa = std::max(kappa, std::fabs(zeta * alpha[s]) * nrm[s]);
      const double inv = nrm[s] > 0 ? 1.0 / nrm[s] : 0.0;
      __half* row = B.data() + (size_t)s * 3 * dp;
      for (int k = 0; k < D; ++k) {
        const double uk = (q_sparse[(size_t)s * D + k] - qbar[k]) * inv;
        const __half hi = __float2half_rn((float)uk);
        const __half lo = __float2half_rn((float)(uk - (double)__half2float(hi)));
        row[k] = hi;
        row[dp + k] = lo;
        row[2 * dp + k] = hi;
        BT[(size_t)k * mp + s] = hi;
      }
    }
    if (!(kappa > 0)) kappa = 1.0;
    for (int s = 0; s < m; ++s) cols[4 * (size_t)s + 3] = (float)(zeta * alpha[s] * nrm[s] / kappa);
    for (int k = 0; k < D; ++k) qb[k] = (float)qbar[k];
    CK(h, ensure(h->tc_B, B.size() * sizeof(__half)));
    CK(h, ensure(h->tc_BT, BT.size() * sizeof(__half)));
    CK(h, ensure(h->tc_cols, cols.size() * sizeof(float)));
    CK(h, ensure(h->tc_qbar, qb.size() * sizeof(float)));
    CK(h, cudaMemcpy(h->tc_B.p, B.data(), B.size() * sizeof(__half), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->tc_BT.p, BT.data(), BT.size() * sizeof(__half), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->tc_cols.p, cols.data(), cols.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->tc_qbar.p, qb.data(), qb.size() * sizeof(float), cudaMemcpyHostToDevice));
    // force-row operand: centred sparse rows scaled by a power of two, two unit columns
    const int dpd = (D + 2 + 63) / 64 * 64;
    double dmax = 0.0;
    for (int s = 0; s < m; ++s)
      for (int k = 0; k < D; ++k) dmax = std::max(dmax, std::fabs(q_sparse[(size_t)s * D + k] - qbar[k]));
    const double kd = dmax > 0 ? std::ldexp(1.0, -std::ilogb(dmax)) : 1.0;
    std::vector<__half> Ad((size_t)mp * dpd, __float2half_rn(0.f));
    for (int s = 0; s < m; ++s) {
      __half* row = Ad.data() + (size_t)s * dpd;
      for (int k = 0; k < D; ++k) row[k] = __float2half_rn((float)(kd * (q_sparse[(size_t)s * D + k] - qbar[k])));
      row[D] = row[D + 1] = __float2half_rn((float)kd);
    }
    CK(h, ensure(h->tc_Ad, Ad.size() * sizeof(__half)));
    CK(h, cudaMemcpy(h->tc_Ad.p, Ad.data(), Ad.size() * sizeof(__half), cudaMemcpyHostToDevice));
    GapTcModel& t = h->tcm;
    t.d = D;
    t.dp = dp;
    t.mp = mp;
    t.izeta = (zeta >= 1.0 && zeta == (double)(int)zeta) ? (int)zeta : 0;
    t.c0 = (float)c0;
    t.zeta = (float)zeta;
    t.kappa = (float)kappa;
    t.B = (const __half*)h->tc_B.p;
    t.BT = (const __half*)h->tc_BT.p;
    t.col = (const float4*)h->tc_cols.p;
    t.qbar = (const float*)h->tc_qbar.p;
    t.dpd = dpd;
    t.kd = (float)kd;
    t.Ad = (const __half*)h->tc_Ad.p;
    t.terms = 3;
    // How much does one FP16 product lose on this model?  The sparse rows, taken as atoms,
    // are environments of the model's own kind: their local energies with one product and
    // with three (~1e-7) give its relative error.  One product is used when that error is
    // at most 1e-5, ten times below the 1e-4 energy bar of the mixed path.
    const int tiles = sg_gap_tc_tiles(mp, t.fwd_cfg);
    CK(h, ensure(h->A16, sizeof(__half) * (size_t)m * 3 * dp));
    CK(h, ensure(h->nrm, sizeof(float) * (size_t)m));
    CK(h, ensure(h->uq, sizeof(float) * (size_t)m));
    CK(h, ensure(h->eps_part, sizeof(float) * (size_t)m * tiles));
    CK(h, ensure(h->r_part, sizeof(float) * (size_t)m * tiles));
    CK(h, ensure(h->err, sizeof(int)));
    CK(h, cudaMemset(h->err.p, 0, sizeof(int)));
    std::vector<double> e_terms[2];
    for (int k = 0; k < 2; ++k) {
      const int terms = k == 0 ? 1 : 3;
      CK(h, sg_gap_tc_prepare((const float*)h->qs.p, m, D, dp, t.qbar, (__half*)h->A16.p, (float*)h->nrm.p,
                              (float*)h->uq.p, terms, 0));
      CK(h, sg_gap_tc_forward(t, terms, (const __half*)h->A16.p, (const float*)h->nrm.p, (const float*)h->uq.p,
                              m, (float*)h->eps_part.p, (float*)h->r_part.p, nullptr, (int*)h->err.p, 0));
      std::vector<float> part((size_t)m * tiles);
      CK(h, cudaMemcpy(part.data(), h->eps_part.p, part.size() * sizeof(float), cudaMemcpyDeviceToHost));
      e_terms[k].assign(m, 0.0);
      for (int s = 0; s < m; ++s)
        for (int j = 0; j < tiles; ++j) e_terms[k][s] += (double)part[(size_t)s * tiles + j];
    }
    int derr = 0;
    CK(h, cudaMemcpy(&derr, h->err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (derr) return fail(h, SOAPGAP_E_CUDA, device_error_text(derr));
    double num = 0.0, den = 0.0;
    for (int s = 0; s < m; ++s) {
      num += (e_terms[0][s] - e_terms[1][s]) * (e_terms[0][s] - e_terms[1][s]);
      den += e_terms[1][s] * e_terms[1][s];
    }
    h->gap_probe_err = den > 0 ? std::sqrt(num / den) : (num > 0 ? 1.0 : 0.0);
    t.terms = h->gap_terms_forced ? h->gap_terms_forced : (h->gap_probe_err <= 1e-5 ? 1 : 3);
  } else {
    CK(h, cudaMemcpy(h->qs.p, q_sparse, nq * es, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->alpha.p, alpha, (size_t)m * es, cudaMemcpyHostToDevice));
  }
  h->M = m;
  h->zeta = zeta;
  h->has_model = true;
  return SOAPGAP_OK;
}

// ---------------------------------------------------------------- geometry set-up
static int setup_geometry(soapgap_handle* h, const soapgap_batch* b) {
  const int S = b->n_struct;
  if ((size_t)S > h->h_geom_cap) {
    if (h->async_call)
      return fail(h, SOAPGAP_E_STATE, "host staging too small for an asynchronous call: make one synchronous call with the same batch first");
    if (h->h_geom) cudaFreeHost(h->h_geom);
    h->h_geom = nullptr;
    h->h_geom_cap = 0;
    CK(h, cudaMallocHost(&h->h_geom, sizeof(StructGeom) * (size_t)S));
    h->h_geom_cap = S;
  }
  const double rc = h->prm.r_cut + h->skin;  // list radius
  int bins = 0, max_atoms = 0;
  double slot_est = 0.0;
  for (int s = 0; s < S; ++s) {
    StructGeom& g = h->h_geom[s];
    const double* c = b->cell_host + 9 * s;
    for (int k = 0; k < 9; ++k) {
      g.h[k] = c[k];
      g.h32[k] = (float)c[k];
      g.h32lo[k] = (float)(c[k] - (double)g.h32[k]);
    }
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    if (!(std::fabs(det) > 0) || !std::isfinite(det))
      return fail(h, SOAPGAP_E_INVALID_ARG, "cell of structure " + std::to_string(s) + " is singular");
    // inverse (rows of h are lattice vectors; fractional = x @ hinv)
    double inv[9] = {c[4] * c[8] - c[5] * c[7], c[2] * c[7] - c[1] * c[8], c[1] * c[5] - c[2] * c[4],
                     c[5] * c[6] - c[3] * c[8], c[0] * c[8] - c[2] * c[6], c[2] * c[3] - c[0] * c[5],
                     c[3] * c[7] - c[4] * c[6], c[1] * c[6] - c[0] * c[7], c[0] * c[4] - c[1] * c[3]};
    for (int k = 0; k < 9; ++k) g.hinv[k] = inv[k] / det;
    const int na = (int)(b->atom_offs_host[s + 1] - b->atom_offs_host[s]);
    double H = 0;
    int mmax = 0;
    for (int k = 0; k < 3; ++k) {
      const double* u = c + 3 * ((k + 1) % 3);
      const double* v = c + 3 * ((k + 2) % 3);
      const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2],
                   cz = u[0] * v[1] - u[1] * v[0];
      const double dk = std::fabs(det) / std::sqrt(cx * cx + cy * cy + cz * cz);
      int nb = (int)std::floor(dk / rc);
      if (nb < 1) nb = 1;
      const int nb_cap = std::max(1, (int)std::cbrt((double)std::max(na, 1)) + 1);
      if (nb > 2 * nb_cap) nb = 2 * nb_cap;  // no more bins than atoms need
      g.nb[k] = nb;
      g.m[k] = (int)std::floor(rc * nb / dk) + 1;
      if (g.m[k] > 100)
        return fail(h, SOAPGAP_E_UNSUPPORTED, "cell too thin for r_cut (more than 100 images)");
      mmax = std::max(mmax, g.m[k]);
      H += std::sqrt(c[3 * k] * c[3 * k] + c[3 * k + 1] * c[3 * k + 1] + c[3 * k + 2] * c[3 * k + 2]);
    }
    const double X = H * (mmax + 3), u = std::ldexp(1.0, -24);
    // |error| of each FP32 separation component <= 10 u X (rounded positions, FP32 shift from
    // rounded lattice vectors, two additions); the margin bounds the error of d2 twice over
    g.margin = (float)(2.0 * (2.0 * std::sqrt(3.0) * 10.0 * rc * X * u + 4.0 * rc * rc * u) + 1e-30);
    max_atoms = std::max(max_atoms, na);
    // kept pairs per atom ~ density x sphere volume (periodic images included)
    const double est = (double)na / std::fabs(det) * 4.18879020478639 * rc * rc * rc;
    slot_est = std::max(slot_est, est);
    g.bin_off = bins;
    g.atom_off = (int)b->atom_offs_host[s];
    g.n_atoms = na;
    bins += g.nb[0] * g.nb[1] * g.nb[2];
  }
  h->n_bins = bins;
  h->finish_chunks = sg_finish_chunks(max_atoms);
  h->slot_maxn_est = ((int)std::ceil(1.3 * slot_est) + 32 + 7) & ~7;
  return SOAPGAP_OK;
}

// structure index of every atom: the last s with offs[s] <= i (skips empty structures)
__global__ void atom_struct_kernel(const int64_t* __restrict__ offs, int S, int n, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  out[i] = lo;
}

__global__ void fill_ones(double* w, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = 1.0;
}

static std::string device_error_text(int code) {
  std::string m;
  if (code & SG_ERR_OUTSIDE_CELL) m += "a position is not finite; ";
  if (code & SG_ERR_COINCIDENT) m += "two atoms coincide (zero separation); ";
  if (code & SG_ERR_PAIR_CAPACITY) m += "pair buffer overflow; ";
  if (code & SG_ERR_NO_REVERSE) m += "pair list not symmetric; ";
  if (code & SG_ERR_TIMEOUT) m += "a tensor-core pipeline wait timed out; ";
  return m;
}

// tuning-table key of a problem class: basis class, species, 32-pair batches per atom (the
// adjoint's shape) and the power of two of the atom count (the GAP products' row tiles)
static long long plan_key(const soapgap_handle* h, int n_atoms, long long n_pairs) {
  const int nsp = h->prm.n_species;
  const int batches = std::min(63, sg_adj_batches_per_atom(n_pairs, n_atoms, nsp));
  int lg = 0;
  while (lg < 31 && (1LL << lg) < (long long)n_atoms) ++lg;
  return (((long long)h->cls * 16 + nsp) * 64 + batches) * 32 + lg;
}

static soapgap_handle::TilePlan plan_for(const soapgap_handle* h, int n_atoms) {
  auto it = h->plans.find(plan_key(h, n_atoms, h->last_pairs));
  return it == h->plans.end() ? soapgap_handle::TilePlan{} : it->second;
}

// arguments of the adjoint pair kernel from the handle's workspace (after a forward pass)
template <typename T>
static AdjArgs<T> adj_args(soapgap_handle* h, int N, const int* species) {
  AdjArgs<T> aa{};
  aa.n_atoms = N; aa.nsp = h->prm.n_species; aa.nmax = h->prm.n_max; aa.lmax = h->prm.l_max;
  aa.dim = h->D;
  aa.n_pairs = h->last_pairs;
  aa.warps = plan_for(h, N).adj_warps;
  aa.species = species; aa.atom_struct = (const int*)h->atom_struct.p;
  aa.struct_w = (const double*)h->struct_w.p;
  aa.list_offs = (const int*)h->seg_offs.p;
  aa.seg_offs = h->skin > 0.0 ? (const int*)h->live_offs.p : (const int*)h->seg_offs.p;
  aa.pair_idx = h->skin > 0.0 ? (const int*)h->live_idx.p : nullptr;
  aa.pair_r = (const Vec4<T>*)h->pair_r.p; aa.table = (const float*)h->table_adj.p; aa.ti = h->ti_adj;
  aa.p = h->dp;
  if constexpr (sizeof(T) == 4) { aa.yc = h->yc32; aa.bc = h->bc32; }
  else { aa.yc = h->yc64; aa.bc = h->bc64; }
  aa.c = (const T*)h->c.p; aa.q = (const T*)h->q.p; aa.pnorm = (const T*)h->pnorm.p;
  aa.g = (const T*)h->g.p; aa.dedr = (Vec4<T>*)h->dedr.p; aa.vir_atom = (T*)h->vir_atom.p;
  aa.err = (int*)h->err.p;
  aa.gimg = (unsigned char*)h->adj_img.p;
  aa.gexp = (int*)h->adj_exp.p;
  return aa;
}

// arguments of the forward pair kernel (after the neighbour list of this batch)
template <typename T>
static FwdArgs<T> fwd_args(soapgap_handle* h, int N, const int* species) {
  FwdArgs<T> fa{};
  fa.n_atoms = N; fa.nsp = h->prm.n_species; fa.nmax = h->prm.n_max; fa.lmax = h->prm.l_max;
  fa.species = species; fa.pair_r = (const Vec4<T>*)h->pair_r.p;
  fa.seg_offs = h->skin > 0.0 ? (const int*)h->live_offs.p : (const int*)h->seg_offs.p;
  fa.pair_idx = h->skin > 0.0 ? (const int*)h->live_idx.p : nullptr;
  fa.table = (const float*)h->table.p; fa.ti = h->ti; fa.p = h->dp;
  if constexpr (sizeof(T) == 4) { fa.yc = h->yc32; fa.bc = h->bc32; }
  else { fa.yc = h->yc64; fa.bc = h->bc64; }
  fa.c = (T*)h->c.p;
  fa.err = (int*)h->err.p;
  fa.mma_sa = h->fwd_sa;
  fa.mma_sb = h->fwd_sb;
  return fa;
}

// the forward pair kernel of tile-plan variant v (mixed path: 1 = FP32 FMA contraction,
// 2 = tensor cores, 0 = the default, FP32 FMA); the FP64 path has one kernel
template <typename T>
static cudaError_t launch_forward(const soapgap_handle* h, const FwdArgs<T>& fa, int v, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (v == 2 && sg_pair_forward_mma_supported(h->cls)) return sg_pair_forward_mma(fa, h->cls, st);
  }
  return sg_pair_forward<T>(fa, h->cls, h->mixed, st);
}

template <typename T>
static int run(soapgap_handle* h, const soapgap_batch* b, uint32_t flags, void* q_out,
               void* pnorm_out, void* e_atom_out, double* e_struct, double* forces,
               double* virial, const double* struct_w_user, double* grad_pos, bool backward,
               cudaStream_t st) {
  const int N = b->n_atoms, S = b->n_struct, nsp = h->prm.n_species;
  const bool want_energy = (flags & (SOAPGAP_ENERGY | SOAPGAP_FORCES | SOAPGAP_VIRIAL)) != 0;
  const bool want_grad = backward || (flags & (SOAPGAP_FORCES | SOAPGAP_VIRIAL)) != 0;
  const size_t es = sizeof(T);
  NbrBuffers nb{};
  const long long launches0 = sg_kernel_launches;
  const size_t N1n = (size_t)std::max(N, 1);
  if (!backward) {
    // the workspace is about to change: until this call succeeds there is no forward pass
    // for soapgap_backward to use
    h->have_forward = false;
    int rc = setup_geometry(h, b);
    if (rc != SOAPGAP_OK) return rc;
    const int nseg = N * nsp;
    ENS(h, h->geom, sizeof(StructGeom) * (size_t)S);
    ENS(h, h->atom_offs, sizeof(int64_t) * (size_t)(S + 1));
    ENS(h, h->atom_struct, sizeof(int) * (size_t)std::max(N, 1));
    ENS(h, h->atom_bin, sizeof(int) * (size_t)std::max(N, 1));
    ENS(h, h->atom_bin4, sizeof(int4) * (size_t)std::max(N, 1));
    ENS(h, h->atom_slot, sizeof(int) * (size_t)std::max(N, 1));
    ENS(h, h->bin_atoms, sizeof(int) * (size_t)std::max(N, 1));
    ENS(h, h->binpos, sizeof(float4) * (size_t)std::max(N, 1));
    ENS(h, h->atom_hi, sizeof(float4) * (size_t)std::max(N, 1));
    ENS(h, h->atom_lo, sizeof(float4) * (size_t)std::max(N, 1));
    ENS(h, h->bin_count, sizeof(int) * (size_t)(h->n_bins + 1));
    ENS(h, h->bin_start, sizeof(int) * (size_t)(h->n_bins + 1));
    ENS(h, h->seg_count, sizeof(int) * (size_t)std::max(nseg, 1));
    ENS(h, h->seg_offs, sizeof(int) * (size_t)(nseg + 1));
    ENS(h, h->scan_tmp, sizeof(int) * sg_scan_tmp_ints(std::max(std::max(nseg, h->n_bins), 1)));
    CK(h, cudaMemcpyAsync(h->geom.p, h->h_geom, sizeof(StructGeom) * (size_t)S, cudaMemcpyHostToDevice, st));
    // atom offsets through pinned staging: a copy captured in a CUDA graph reads it at replay
    if ((size_t)(S + 1) > h->h_offs_cap) {
      if (h->async_call)
        return fail(h, SOAPGAP_E_STATE, "host staging too small for an asynchronous call: make one synchronous call with the same batch first");
      if (h->h_offs) cudaFreeHost(h->h_offs);
      h->h_offs = nullptr;
      h->h_offs_cap = 0;
      CK(h, cudaMallocHost(&h->h_offs, sizeof(int64_t) * (size_t)(S + 1)));
      h->h_offs_cap = (size_t)(S + 1);
    }
    std::memcpy(h->h_offs, b->atom_offs_host, sizeof(int64_t) * (size_t)(S + 1));
    CK(h, cudaMemcpyAsync(h->atom_offs.p, h->h_offs, sizeof(int64_t) * (size_t)(S + 1),
                          cudaMemcpyHostToDevice, st));
    CK(h, cudaMemsetAsync(h->err.p, 0, sizeof(int), st));
    mark(h, EV_NB0, st);
    if (N > 0)
      atom_struct_kernel<<<(N + 255) / 256, 256, 0, st>>>((const int64_t*)h->atom_offs.p, S, N,
                                                           (int*)h->atom_struct.p);
    ++sg_kernel_launches;
  }
  nb.geom = (const StructGeom*)h->geom.p;
  nb.atom_struct = (const int*)h->atom_struct.p;
  nb.atom_bin = (int*)h->atom_bin.p;
  nb.atom_bin4 = (int4*)h->atom_bin4.p;
  nb.atom_slot = (int*)h->atom_slot.p;
  nb.bin_count = (int*)h->bin_count.p;
  nb.bin_start = (int*)h->bin_start.p;
  nb.bin_atoms = (int*)h->bin_atoms.p;
  nb.binpos = (float4*)h->binpos.p;
  nb.atom_hi = (float4*)h->atom_hi.p;
  nb.atom_lo = (float4*)h->atom_lo.p;
  nb.seg_count = (int*)h->seg_count.p;
  nb.seg_offs = (int*)h->seg_offs.p;
  nb.scan_tmp = (int*)h->scan_tmp.p;
  nb.err = (int*)h->err.p;
  nb.run = nullptr;
  nb.rc2_mask = h->skin > 0.0 ? h->prm.r_cut * h->prm.r_cut : 0.0;
  nb.n_struct = S;
  nb.n_bins = h->n_bins;
  nb.sweep = plan_for(h, N).nbr_sweep;
  // Verlet skin: reuse the list while no atom has moved by skin/2 since its build
  bool rebuild = true, device_decides = false;
  if (!backward && h->skin > 0.0) {
    ENS(h, h->skin_flag, sizeof(int));
    ENS(h, h->pos_ref, sizeof(double) * 3 * N1n);
    const bool same = h->ref_valid && h->ref_atoms == N && h->ref_struct == S &&
                      h->ref_cell.size() == (size_t)9 * S &&
                      std::memcmp(h->ref_cell.data(), b->cell_host, sizeof(double) * 9 * S) == 0;
    if (same) {
      CK(h, cudaMemsetAsync(h->skin_flag.p, 0, sizeof(int), st));
      CK(h, sg_skin_check(b->pos, (const double*)h->pos_ref.p, N, 0.5 * h->skin, (int*)h->skin_flag.p, st));
      if (h->async_call) {
        device_decides = true;
        nb.run = (const int*)h->skin_flag.p;
      } else {
        CK(h, cudaMemcpyAsync(h->h_count, h->skin_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(h, cudaStreamSynchronize(st));
        rebuild = h->h_count[0] != 0;
      }
    } else if (h->async_call) {
      return fail(h, SOAPGAP_E_STATE, "no neighbour list to reuse for an asynchronous call: make one synchronous call with the same batch first");
    }
  }
  h->last_rebuild = device_decides ? -1 : (rebuild ? 1 : 0);
  if (!backward && (rebuild || device_decides)) {
    // one sweep over the candidates into per-atom slot arrays; a synchronous call retries
    // once with the measured largest count if the density estimate was too small
    int maxn = h->async_call ? h->slot_maxn : h->slot_maxn_est;
    // a rebuild overwrites the list: it may be reused or exported only once it completes
    // (an asynchronous rebuild never reads its pair count back, so it does not count)
    if (!device_decides) h->ref_valid = false;
    h->list_ok = false;
    if (h->async_call && maxn <= 0)
      return fail(h, SOAPGAP_E_STATE, "no neighbour slots for an asynchronous call: make one synchronous call with the same batch first");
    ENS(h, h->slot_count, sizeof(int) * N1n);
    ENS(h, h->max_count, sizeof(int));
    ENS(h, h->pos_w, sizeof(double) * 3 * N1n);
    ENS(h, h->img, sizeof(int4) * N1n);
    nb.slot_count = (int*)h->slot_count.p;
    nb.max_count = (int*)h->max_count.p;
    // the list is built from the positions mapped into their cells (identical for atoms
    // already inside)
    CK(h, sg_nbr_wrap(b->pos, N, nb, (double*)h->pos_w.p, (int4*)h->img.p, st));
    CK(h, sg_nbr_bin((const double*)h->pos_w.p, b->species, N, h->n_bins, nb, st));
    for (int attempt = 0; attempt < 2; ++attempt) {
      // pair offsets are 32-bit: a sweep that raises no capacity flag has at most maxn pairs
      // per atom, so N maxn below 2^31 keeps every offset and the total in range
      if ((long long)N * maxn > 0x7fffffffLL)
        return fail(h, SOAPGAP_E_UNSUPPORTED,
                    "too many neighbour pairs for 32-bit pair offsets (atoms x per-atom slots >= 2^31): split the batch");
      ENS(h, h->key_tmp, 8 * N1n * (size_t)maxn);
      nb.key_tmp = (unsigned long long*)h->key_tmp.p;
      CK(h, sg_nbr_slots((const double*)h->pos_w.p, b->species, N, nsp, h->prm.r_cut + h->skin, maxn, nb, st));
      if (h->async_call) break;
      CK(h, cudaMemcpyAsync(h->h_count, (int*)h->seg_offs.p + N * nsp, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(h, cudaMemcpyAsync(h->h_count + 1, h->max_count.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(h, cudaMemcpyAsync(h->h_err, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(h, cudaStreamSynchronize(st));
      const int derr = *h->h_err;
      if (derr & ~SG_ERR_PAIR_CAPACITY) return fail(h, SOAPGAP_E_INVALID_ARG, device_error_text(derr));
      if (h->h_count[1] > maxn && attempt == 0) {
        maxn = (h->h_count[1] + 8 + 7) & ~7;
        CK(h, cudaMemsetAsync(h->err.p, 0, sizeof(int), st));
        continue;
      }
      if (derr) return fail(h, SOAPGAP_E_INVALID_ARG, device_error_text(derr));
      h->last_pairs = *h->h_count;
      h->slot_maxn = maxn;
      break;
    }
    h->cur_maxn = maxn;
    mark(h, EV_NB1, st);
  }
  long long P = h->last_pairs;
  if (h->async_call && !backward) {  // (with a skin, the guard itself runs only on rebuilds)
    // the pair count is not read back: the pair buffers' capacity bounds it, and a
    // device-side guard empties every segment (and flags SG_ERR_PAIR_CAPACITY) if the
    // count exceeds it or a slot array overflowed
    const Buf* pb[4] = {&h->key, &h->pair_j, &h->pair_r, &h->rev};
    const size_t el[4] = {8, 4, sizeof(Vec4<T>), 4};
    long long cap = std::numeric_limits<long long>::max();
    for (int k = 0; k < 4; ++k) {
      if (!pb[k]->p) return fail(h, SOAPGAP_E_STATE, "no pair buffers for an asynchronous call: make one synchronous call with the same batch first");
      cap = std::min(cap, (long long)(pb[k]->cap / el[k]));
    }
    if (want_grad) {
      if (!h->dedr.p) return fail(h, SOAPGAP_E_STATE, "no pair buffers for an asynchronous call: make one synchronous call with the same batch first");
      cap = std::min(cap, (long long)(h->dedr.cap / sizeof(Vec4<T>)));
    }
    if (h->skin > 0.0) {
      if (!h->live_idx.p) return fail(h, SOAPGAP_E_STATE, "no pair buffers for an asynchronous call: make one synchronous call with the same batch first");
      cap = std::min(cap, (long long)(h->live_idx.cap / sizeof(int)));
    }
    P = cap;
    CK(h, sg_nbr_cap_guard((int*)h->seg_offs.p, N * nsp, P, (int*)h->err.p, st, nb.run));
  }
  const size_t Pc = (size_t)std::max(P, 1LL);
  ENS(h, h->key, 8 * Pc);
  ENS(h, h->pair_j, 4 * Pc);
  ENS(h, h->pair_r, sizeof(Vec4<T>) * Pc);
  ENS(h, h->rev, 4 * Pc);
  nb.key_tmp = (unsigned long long*)h->key_tmp.p;
  nb.slot_count = (int*)h->slot_count.p;
  nb.max_count = (int*)h->max_count.p;
  nb.key = (unsigned long long*)h->key.p;
  nb.pair_j = (int*)h->pair_j.p;
  nb.pair_r = h->pair_r.p;
  nb.rev = (int*)h->rev.p;
  const int L = h->L, nch = h->nch, D = h->D;
  const size_t N1 = (size_t)std::max(N, 1);
  ENS(h, h->c, es * N1 * nch * L);
  ENS(h, h->q, es * N1 * D);
  ENS(h, h->pnorm, es * N1);
  bool fused_operand = false;  // A16 / nrm / uq written by the power-spectrum kernel
  if (!backward) {
    mark(h, EV_FILL0, st);
    if (rebuild || device_decides) {
      cudaError_t e = sg_nbr_place<T>((const double*)h->pos_w.p, b->species, N, nsp, h->cur_maxn, nb, st);
      if (e == cudaErrorInvalidConfiguration)
        return fail(h, SOAPGAP_E_UNSUPPORTED, "too many neighbours per atom for the pair sort");
      CK(h, e);
      if (!h->async_call) {
        h->list_ok = true;
        h->list_atoms = N;
      }
    }
    if (h->skin > 0.0) {
      // every call: current separations of the whole list and the list of live pairs
      // (within r_cut), which the pair kernels and the force gather then use
      ENS(h, h->live_count, sizeof(int) * N1n * nsp);
      ENS(h, h->live_offs, sizeof(int) * (N1n * nsp + 1));
      ENS(h, h->live_idx, sizeof(int) * Pc);
      NbrBuffers nr = nb;  // positions as given, with the cell images of the last build
      nr.img = (const int4*)h->img.p;
      nr.run = nullptr;
      CK(h, sg_nbr_refresh<T>(b->pos, N, nsp, nr, (int*)h->live_count.p, (int*)h->live_offs.p,
                              (int*)h->live_idx.p, st));
      if (device_decides) {
        CK(h, sg_skin_ref_update(b->pos, (double*)h->pos_ref.p, N, (const int*)h->skin_flag.p, st));
      } else if (rebuild) {
        CK(h, cudaMemcpyAsync(h->pos_ref.p, b->pos, sizeof(double) * 3 * (size_t)N, cudaMemcpyDeviceToDevice, st));
        h->ref_valid = true;
        h->ref_atoms = N;
        h->ref_struct = S;
        h->ref_cell.assign(b->cell_host, b->cell_host + 9 * (size_t)S);
      }
    }
    mark(h, EV_FWD0, st);
    h->stage_ran[0] = h->stage_ran[1] = h->stage_ran[2] = true;
    const FwdArgs<T> fa = fwd_args<T>(h, N, b->species);
    CK(h, launch_forward<T>(h, fa, plan_for(h, N).pair_fwd, st));
    mark(h, EV_PS0, st);
    GapOperand op{};
    if constexpr (sizeof(T) == 4) {
      if (want_energy) {
        // the tensor-core GAP operand of each atom is written by the power-spectrum kernel
        const GapTcModel& tm = h->tcm;
        ENS(h, h->A16, sizeof(__half) * N1 * tm.terms * tm.dp);
        ENS(h, h->nrm, sizeof(float) * N1);
        ENS(h, h->uq, sizeof(float) * N1);
        op = GapOperand{(__half*)h->A16.p, (float*)h->nrm.p, (float*)h->uq.p, tm.qbar, tm.dp, tm.terms};
        fused_operand = true;
      }
    }
    CK(h, sg_power_spectrum<T>((const T*)h->c.p, N, nch, h->prm.l_max, h->LC, (T*)h->q.p, (T*)h->pnorm.p, st, op));
    if ((flags & SOAPGAP_DESC) && q_out)
      CK(h, cudaMemcpyAsync(q_out, h->q.p, es * (size_t)N * D, cudaMemcpyDeviceToDevice, st));
    if ((flags & SOAPGAP_DESC) && pnorm_out)
      CK(h, cudaMemcpyAsync(pnorm_out, h->pnorm.p, es * (size_t)N, cudaMemcpyDeviceToDevice, st));
  }
  if (want_energy || backward) {
    const int M = h->M;
    GapTcModel tm = h->tcm;  // with the tile configurations of this problem class
    if (h->mixed) {
      const soapgap_handle::TilePlan pl = plan_for(h, N);
      tm.fwd_cfg = pl.gap_fwd;
      tm.bwd_cfg = pl.gap_bwd;
    }
    const int tiles = h->mixed ? sg_gap_tc_tiles(tm.mp, tm.fwd_cfg) : sg_gap_tiles(M);
    const int tiles_alloc = h->mixed ? sg_gap_tc_tiles_max(tm.mp) : tiles;
    ENS(h, h->eps_part, es * N1 * tiles_alloc);
    ENS(h, h->e_atom, es * N1);
    if (want_grad) {
      if (!h->mixed) ENS(h, h->kp, es * N1 * M);
      ENS(h, h->g, es * N1 * D);
      ENS(h, h->vir_atom, es * N1 * 9);
      ENS(h, h->dedr, sizeof(Vec4<T>) * Pc);
      if (h->mixed) {
        ENS(h, h->adj_img, sg_adj_tc_image_bytes(h->cls, nsp) * N1);
        ENS(h, h->adj_exp, sizeof(int) * N1);
      }
      ENS(h, h->struct_w, sizeof(double) * (size_t)S);
    }
    mark(h, EV_GF0, st);
    h->stage_ran[3] = true;
    if constexpr (sizeof(T) == 4) {
      // tensor cores: centred, norm-scaled FP16 split operands (see gap_tc.cu)
      ENS(h, h->A16, sizeof(__half) * N1 * tm.terms * tm.dp);
      ENS(h, h->nrm, sizeof(float) * N1);
      ENS(h, h->uq, sizeof(float) * N1);
      ENS(h, h->r_part, sizeof(float) * N1 * tiles_alloc);
      if (want_grad) ENS(h, h->kp16, sizeof(__half) * N1 * tm.mp);
      if (!fused_operand)
        CK(h, sg_gap_tc_prepare((const float*)h->q.p, N, D, tm.dp, tm.qbar, (__half*)h->A16.p,
                                (float*)h->nrm.p, (float*)h->uq.p, tm.terms, st));
      CK(h, sg_gap_tc_forward(tm, tm.terms, (const __half*)h->A16.p, (const float*)h->nrm.p, (const float*)h->uq.p, N,
                              (float*)h->eps_part.p, (float*)h->r_part.p,
                              want_grad ? (__half*)h->kp16.p : nullptr, (int*)h->err.p, st));
    } else {
      CK(h, sg_gap_forward_simt<T>((const T*)h->q.p, (const T*)h->qs.p, (const T*)h->alpha.p, N, M, D,
                                   h->zeta, (T*)h->eps_part.p, tiles, want_grad ? (T*)h->kp.p : nullptr, st));
    }
    mark(h, EV_GB0, st);
    if (want_grad) {
      h->stage_ran[4] = h->stage_ran[5] = true;
      if constexpr (sizeof(T) == 4)
        CK(h, sg_gap_tc_backward(tm, (const __half*)h->kp16.p, (const float*)h->r_part.p, N,
                                 (float*)h->g.p, (int*)h->err.p, st));
      else
        CK(h, sg_gap_backward_simt<T>((const T*)h->kp.p, (const T*)h->qs.p, N, M, D, (T*)h->g.p, st));
      if (struct_w_user) {
        CK(h, cudaMemcpyAsync(h->struct_w.p, struct_w_user, sizeof(double) * S, cudaMemcpyDeviceToDevice, st));
      } else {
        fill_ones<<<(S + 255) / 256, 256, 0, st>>>((double*)h->struct_w.p, S);
        ++sg_kernel_launches;
      }
      AdjArgs<T> aa = adj_args<T>(h, N, b->species);
      mark(h, EV_ADJ0, st);
      cudaError_t e = sg_pair_adjoint<T>(aa, h->cls, h->mixed, st);
      if (e == cudaErrorInvalidConfiguration)
        return fail(h, SOAPGAP_E_UNSUPPORTED, "descriptor too large for the adjoint kernel's shared memory");
      CK(h, e);
    }
    mark(h, EV_FIN0, st);
    h->stage_ran[6] = true;
    double* f_out = backward ? grad_pos : ((flags & SOAPGAP_FORCES) ? forces : nullptr);
    double* v_out = (backward || (flags & SOAPGAP_VIRIAL)) ? virial : nullptr;
    double* es_out = backward ? nullptr : e_struct;
    ENS(h, h->finish_part, sizeof(double) * 10 * (size_t)S * h->finish_chunks);
    CK(h, sg_finish<T>(N, S, nsp, (const int64_t*)h->atom_offs.p,
                       h->skin > 0.0 ? (const int*)h->live_offs.p : nb.seg_offs,
                       h->skin > 0.0 ? (const int*)h->live_idx.p : nullptr, (const int*)h->rev.p,
                       (const Vec4<T>*)h->dedr.p, (const T*)h->eps_part.p, tiles,
                       v_out ? (const T*)h->vir_atom.p : nullptr, (T*)h->e_atom.p, es_out, f_out,
                       v_out, !backward, h->finish_chunks, (double*)h->finish_part.p, st));
    if (!backward && e_atom_out)
      CK(h, cudaMemcpyAsync(e_atom_out, h->e_atom.p, es * (size_t)N, cudaMemcpyDeviceToDevice, st));
  }
  mark(h, EV_END, st);
  if (h->async_call) {
    // no synchronisation: the error word lands in pinned memory for soapgap_sync_status
    CK(h, cudaMemcpyAsync(h->h_err_async, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    h->launches = sg_kernel_launches - launches0;
    if (!backward) {
      h->have_forward = want_energy;
      h->fw_atoms = N;
      h->fw_struct = S;
    }
    h->msg.clear();
    return SOAPGAP_OK;
  }
  CK(h, cudaMemcpyAsync(h->h_err, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  h->launches = sg_kernel_launches - launches0;
  if (*h->h_err) return fail(h, SOAPGAP_E_INVALID_ARG, device_error_text(*h->h_err));
  if (!backward) {
    h->have_forward = want_energy;
    h->fw_atoms = N;
    h->fw_struct = S;
  }
  h->msg.clear();
  return SOAPGAP_OK;
}

static int check_batch(soapgap_handle* h, const soapgap_batch* b) {
  if (!b) return fail(h, SOAPGAP_E_INVALID_ARG, "batch is NULL");
  if (b->n_struct < 1 || b->n_atoms < 0) return fail(h, SOAPGAP_E_INVALID_ARG, "need n_struct >= 1 and n_atoms >= 0");
  if (!b->atom_offs_host || !b->cell_host) return fail(h, SOAPGAP_E_INVALID_ARG, "atom_offs_host and cell_host are required");
  if (b->atom_offs_host[0] != 0 || b->atom_offs_host[b->n_struct] != b->n_atoms)
    return fail(h, SOAPGAP_E_INVALID_ARG, "atom_offs_host must start at 0 and end at n_atoms");
  for (int s = 0; s < b->n_struct; ++s)
    if (b->atom_offs_host[s + 1] < b->atom_offs_host[s]) return fail(h, SOAPGAP_E_INVALID_ARG, "atom_offs_host must be nondecreasing");
  if (b->n_atoms > 0 && (!b->pos || !b->species)) return fail(h, SOAPGAP_E_INVALID_ARG, "pos and species are required");
  if ((long long)b->n_atoms * h->prm.n_species >= (1LL << 30) || b->n_atoms >= (1 << 28))
    return fail(h, SOAPGAP_E_UNSUPPORTED, "too many atoms");
  return SOAPGAP_OK;
}

extern "C" int soapgap_compute(soapgap_handle* h, const soapgap_batch* batch, uint32_t flags,
                               void* q, void* pnorm, void* e_atom, double* e_struct, double* forces,
                               double* virial, void* stream) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  int rc = check_batch(h, batch);
  if (rc != SOAPGAP_OK) return rc;
  if (flags & ~(SOAPGAP_DESC | SOAPGAP_ENERGY | SOAPGAP_FORCES | SOAPGAP_VIRIAL | SOAPGAP_TIMING |
                SOAPGAP_ASYNC))
    return fail(h, SOAPGAP_E_INVALID_ARG, "unknown flag bits");
  if ((flags & SOAPGAP_ASYNC) && (flags & SOAPGAP_TIMING))
    return fail(h, SOAPGAP_E_INVALID_ARG, "SOAPGAP_TIMING cannot be combined with SOAPGAP_ASYNC");
  h->async_call = (flags & SOAPGAP_ASYNC) != 0;
  h->timed = (flags & SOAPGAP_TIMING) != 0;
  for (int k = 0; k < SOAPGAP_N_STAGES; ++k) h->stage_ran[k] = false;
  if (h->timed && !h->ev_made) {
    for (int k = 0; k < 10; ++k) CK(h, cudaEventCreate(&h->ev[k]));
    h->ev_made = true;
  }
  if ((flags & SOAPGAP_DESC) && !q) return fail(h, SOAPGAP_E_INVALID_ARG, "DESC needs q");
  if ((flags & SOAPGAP_ENERGY) && (!e_struct && !e_atom)) return fail(h, SOAPGAP_E_INVALID_ARG, "ENERGY needs e_struct or e_atom");
  if ((flags & SOAPGAP_FORCES) && !forces) return fail(h, SOAPGAP_E_INVALID_ARG, "FORCES needs forces");
  if ((flags & SOAPGAP_VIRIAL) && !virial) return fail(h, SOAPGAP_E_INVALID_ARG, "VIRIAL needs virial");
  if ((flags & (SOAPGAP_ENERGY | SOAPGAP_FORCES | SOAPGAP_VIRIAL)) && !h->has_model)
    return fail(h, SOAPGAP_E_STATE, "no GAP model: call soapgap_set_model first");
  if (!(flags & SOAPGAP_DESC)) { q = nullptr; pnorm = nullptr; }
  cudaStream_t st = (cudaStream_t)stream;
  if (h->mixed)
    return run<float>(h, batch, flags, q, pnorm, e_atom, e_struct, forces, virial, nullptr, nullptr, false, st);
  return run<double>(h, batch, flags, q, pnorm, e_atom, e_struct, forces, virial, nullptr, nullptr, false, st);
}

extern "C" int soapgap_backward(soapgap_handle* h, const soapgap_batch* batch, const double* dE_dEstruct,
                                double* grad_pos, double* virial, void* stream) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  int rc = check_batch(h, batch);
  if (rc != SOAPGAP_OK) return rc;
  if (!h->has_model) return fail(h, SOAPGAP_E_STATE, "no GAP model: call soapgap_set_model first");
  if (!h->have_forward || h->fw_atoms != batch->n_atoms || h->fw_struct != batch->n_struct)
    return fail(h, SOAPGAP_E_STATE, "backward needs a preceding ENERGY evaluation of the same batch");
  if (!dE_dEstruct || !grad_pos) return fail(h, SOAPGAP_E_INVALID_ARG, "backward needs dE_dEstruct and grad_pos");
  cudaStream_t st = (cudaStream_t)stream;
  h->timed = false;
  h->async_call = false;
  if (h->mixed)
    return run<float>(h, batch, 0, nullptr, nullptr, nullptr, nullptr, nullptr, virial, dE_dEstruct, grad_pos, true, st);
  return run<double>(h, batch, 0, nullptr, nullptr, nullptr, nullptr, nullptr, virial, dE_dEstruct, grad_pos, true, st);
}

extern "C" int soapgap_compute_host(soapgap_handle* h, const soapgap_batch* batch, uint32_t flags,
                                    void* q, void* pnorm, void* e_atom, double* e_struct,
                                    double* forces, double* virial, void* stream) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  int rc = check_batch(h, batch);
  if (rc != SOAPGAP_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int N = batch->n_atoms, S = batch->n_struct, D = h->D;
  const size_t es = h->mixed ? sizeof(float) : sizeof(double);
  const size_t N1 = (size_t)std::max(N, 1);
  CK(h, ensure(h->host_in_pos, sizeof(double) * 3 * N1));
  CK(h, ensure(h->host_in_species, sizeof(int) * N1));
  CK(h, cudaMemcpyAsync(h->host_in_pos.p, batch->pos, sizeof(double) * 3 * (size_t)N, cudaMemcpyHostToDevice, st));
  CK(h, cudaMemcpyAsync(h->host_in_species.p, batch->species, sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, st));
  soapgap_batch db = *batch;
  db.pos = (const double*)h->host_in_pos.p;
  db.species = (const int32_t*)h->host_in_species.p;
  void *dq = nullptr, *dpn = nullptr, *dea = nullptr;
  double *des = nullptr, *df = nullptr, *dv = nullptr;
  if (q) { CK(h, ensure(h->host_q, es * N1 * D)); dq = h->host_q.p; }
  if (pnorm) { CK(h, ensure(h->host_pnorm, es * N1)); dpn = h->host_pnorm.p; }
  if (e_atom) { CK(h, ensure(h->host_e_atom, es * N1)); dea = h->host_e_atom.p; }
  if (e_struct) { CK(h, ensure(h->host_e_struct, sizeof(double) * S)); des = (double*)h->host_e_struct.p; }
  if (forces) { CK(h, ensure(h->host_forces, sizeof(double) * 3 * N1)); df = (double*)h->host_forces.p; }
  if (virial) { CK(h, ensure(h->host_virial, sizeof(double) * 9 * S)); dv = (double*)h->host_virial.p; }
  rc = soapgap_compute(h, &db, flags & ~SOAPGAP_ASYNC, dq, dpn, dea, des, df, dv, stream);
  if (rc != SOAPGAP_OK) return rc;
  if (q && (flags & SOAPGAP_DESC)) CK(h, cudaMemcpyAsync(q, dq, es * (size_t)N * D, cudaMemcpyDeviceToHost, st));
  if (pnorm && (flags & SOAPGAP_DESC)) CK(h, cudaMemcpyAsync(pnorm, dpn, es * (size_t)N, cudaMemcpyDeviceToHost, st));
  if (e_atom && (flags & SOAPGAP_ENERGY)) CK(h, cudaMemcpyAsync(e_atom, dea, es * (size_t)N, cudaMemcpyDeviceToHost, st));
  if (e_struct && (flags & SOAPGAP_ENERGY)) CK(h, cudaMemcpyAsync(e_struct, des, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
  if (forces && (flags & SOAPGAP_FORCES)) CK(h, cudaMemcpyAsync(forces, df, sizeof(double) * 3 * (size_t)N, cudaMemcpyDeviceToHost, st));
  if (virial && (flags & SOAPGAP_VIRIAL)) CK(h, cudaMemcpyAsync(virial, dv, sizeof(double) * 9 * S, cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  return SOAPGAP_OK;
}

extern "C" int soapgap_tc_gemm_f16(soapgap_handle* h, const void* a, int32_t m, const void* b, int32_t n,
                                   int32_t k, float* c, void* stream) {
  if (!h || !a || !b || !c || m < 1 || n < 1 || k < 64 || k % 64 != 0) return SOAPGAP_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(h, cudaMemsetAsync(h->err.p, 0, sizeof(int), st));
  CK(h, sg_tc_gemm_store((const __half*)a, m, (const __half*)b, n, k, c, (int*)h->err.p, st));
  CK(h, cudaMemcpyAsync(h->h_err, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if (*h->h_err) return fail(h, SOAPGAP_E_CUDA, device_error_text(*h->h_err));
  return SOAPGAP_OK;
}

extern "C" int soapgap_stage_times(const soapgap_handle* h, double* ms) {
  if (!h || !ms) return SOAPGAP_E_INVALID_ARG;
  if (!h->timed) return SOAPGAP_E_STATE;
  auto span = [&](int a, int b) {
    float t = 0.f;
    return cudaEventElapsedTime(&t, h->ev[a], h->ev[b]) == cudaSuccess ? (double)t : 0.0;
  };
  for (int k = 0; k < SOAPGAP_N_STAGES; ++k) ms[k] = 0.0;
  if (h->stage_ran[0]) ms[0] = span(EV_NB0, EV_NB1) + span(EV_FILL0, EV_FWD0);
  if (h->stage_ran[1]) ms[1] = span(EV_FWD0, EV_PS0);
  if (h->stage_ran[2]) ms[2] = span(EV_PS0, h->stage_ran[3] ? EV_GF0 : EV_END);
  if (h->stage_ran[3]) ms[3] = span(EV_GF0, EV_GB0);
  if (h->stage_ran[4]) ms[4] = span(EV_GB0, EV_ADJ0);
  if (h->stage_ran[5]) ms[5] = span(EV_ADJ0, EV_FIN0);
  if (h->stage_ran[6]) ms[6] = span(h->stage_ran[4] ? EV_FIN0 : EV_GB0, EV_END);
  return SOAPGAP_OK;
}

extern "C" int soapgap_last_launch_count(const soapgap_handle* h, int64_t* n) {
  if (!h || !n) return SOAPGAP_E_INVALID_ARG;
  *n = h->launches;
  return SOAPGAP_OK;
}

extern "C" int soapgap_last_pair_count(const soapgap_handle* h, int64_t* n) {
  if (!h || !n) return SOAPGAP_E_INVALID_ARG;
  *n = h->last_pairs;
  return SOAPGAP_OK;
}

extern "C" int soapgap_export_pairs(soapgap_handle* h, int64_t capacity, int32_t* centre,
                                    int32_t* neighbour, int32_t* shift) {
  if (!h || !centre || !neighbour || !shift) return SOAPGAP_E_INVALID_ARG;
  if (!h->list_ok)
    return fail(h, SOAPGAP_E_STATE, "export_pairs: no complete pair list (the last list build failed or was asynchronous)");
  const long long P = h->last_pairs;
  if (capacity < P) return fail(h, SOAPGAP_E_CAPACITY, "export_pairs: arrays shorter than the pair count");
  if (P == 0) return SOAPGAP_OK;
  const int N = h->list_atoms, nsp = h->prm.n_species;
  std::vector<int> offs((size_t)N * nsp + 1);
  std::vector<unsigned long long> keys((size_t)P);
  CK(h, cudaMemcpy(offs.data(), h->seg_offs.p, sizeof(int) * offs.size(), cudaMemcpyDeviceToHost));
  CK(h, cudaMemcpy(keys.data(), h->key.p, 8 * (size_t)P, cudaMemcpyDeviceToHost));
  // the offsets must span exactly [0, P) in order before they index the caller's arrays
  if (offs[0] != 0 || offs.back() != P) return fail(h, SOAPGAP_E_STATE, "export_pairs: pair offsets inconsistent");
  for (size_t k = 1; k < offs.size(); ++k)
    if (offs[k] < offs[k - 1]) return fail(h, SOAPGAP_E_STATE, "export_pairs: pair offsets inconsistent");
  for (int i = 0; i < N; ++i)
    for (int p = offs[(size_t)i * nsp]; p < offs[(size_t)(i + 1) * nsp]; ++p) centre[p] = i;
  for (long long p = 0; p < P; ++p) {
    const unsigned long long k = keys[p];
    neighbour[p] = (int32_t)(k >> 24);
    shift[3 * p] = (int)((k >> 16) & 255) - 128;
    shift[3 * p + 1] = (int)((k >> 8) & 255) - 128;
    shift[3 * p + 2] = (int)(k & 255) - 128;
  }
  return SOAPGAP_OK;
}

extern "C" const char* soapgap_last_error(const soapgap_handle* h) {
  return h ? h->msg.c_str() : "NULL handle";
}

extern "C" void soapgap_destroy(soapgap_handle* h) {
  if (!h) return;
  Buf* bufs[] = {&h->tc_B, &h->tc_BT, &h->tc_cols, &h->tc_qbar, &h->tc_Ad, &h->A16, &h->nrm, &h->uq,
                 &h->r_part, &h->kp16, &h->table, &h->table_adj, &h->qs, &h->alpha, &h->geom, &h->atom_offs, &h->atom_struct,
                 &h->atom_bin, &h->atom_bin4, &h->atom_slot, &h->bin_count, &h->bin_start, &h->bin_atoms,
                 &h->binpos, &h->atom_hi, &h->atom_lo, &h->seg_count, &h->seg_offs, &h->scan_tmp, &h->key_tmp,
                 &h->key, &h->pair_j, &h->pair_r, &h->rev, &h->dedr, &h->adj_img, &h->adj_exp, &h->c, &h->q, &h->pnorm,
                 &h->e_atom, &h->eps_part, &h->kp, &h->g, &h->vir_atom, &h->struct_w, &h->err,
                 &h->finish_part, &h->slot_count, &h->max_count, &h->pos_ref, &h->skin_flag, &h->live_count, &h->live_offs, &h->live_idx, &h->pos_w, &h->img,
                 &h->cen_tmp, &h->host_in_pos, &h->host_in_species, &h->host_q, &h->host_pnorm,
                 &h->host_e_atom, &h->host_e_struct, &h->host_forces, &h->host_virial,
                 &h->dk_k, &h->dk_wv, &h->dk_J, &h->dk_at, &h->dk_v};
  for (Buf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->h_count) cudaFreeHost(h->h_count);
  if (h->h_geom) cudaFreeHost(h->h_geom);
  if (h->h_offs) cudaFreeHost(h->h_offs);
  if (h->h_err_async) cudaFreeHost(h->h_err_async);
  if (h->ev_made)
    for (int k = 0; k < 10; ++k) cudaEventDestroy(h->ev[k]);
  if (h->dev_made)
    for (int k = 0; k <= SOAPGAP_N_DESIGN_STAGES; ++k) cudaEventDestroy(h->dev_ev[k]);
  delete h;
}

extern "C" int soapgap_sync_status(soapgap_handle* h, void* stream) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  CK(h, cudaStreamSynchronize((cudaStream_t)stream));
  const int code = *h->h_err_async;
  if (!code) {
    h->msg.clear();
    return SOAPGAP_OK;
  }
  const int rc = (code & SG_ERR_PAIR_CAPACITY) ? SOAPGAP_E_CAPACITY
                 : (code & SG_ERR_TIMEOUT)     ? SOAPGAP_E_CUDA
                                               : SOAPGAP_E_INVALID_ARG;
  return fail(h, rc, device_error_text(code));
}

#define TL(x)                          \
  do {                                 \
    const int rc_ = (x);               \
    if (rc_ != SOAPGAP_OK) return rc_; \
  } while (0)

// CUDA-event time (ms) of `launch`, mean of `reps` launches after one untimed launch (which
// also sets kernel attributes and warms the caches); a negative time if it cannot run.
template <typename F>
static int time_launches(soapgap_handle* h, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps,
                         F&& launch, float* ms) {
  float total = 0.f;
  for (int rep = 0; rep <= reps; ++rep) {
    CK(h, cudaEventRecord(e0, st));
    cudaError_t e = launch();
    if (e == cudaErrorInvalidConfiguration) {
      cudaGetLastError();
      *ms = -1.f;
      return SOAPGAP_OK;
    }
    CK(h, e);
    CK(h, cudaEventRecord(e1, st));
    CK(h, cudaEventSynchronize(e1));
    float t = 0.f;
    CK(h, cudaEventElapsedTime(&t, e0, e1));
    if (rep > 0) total += t;
  }
  *ms = total / reps;
  return SOAPGAP_OK;
}

extern "C" int soapgap_autotune(soapgap_handle* h, const soapgap_batch* batch, int32_t* plan,
                                void* stream) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  int rc = check_batch(h, batch);
  if (rc != SOAPGAP_OK) return rc;
  if (!h->has_model) return fail(h, SOAPGAP_E_STATE, "no GAP model: call soapgap_set_model first");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = batch->n_atoms, S = batch->n_struct;
  const size_t N1 = (size_t)std::max(N, 1);
  // one synchronous evaluation sizes the workspace and leaves every stage's inputs
  CK(h, ensure(h->host_e_struct, sizeof(double) * S));
  CK(h, ensure(h->host_forces, sizeof(double) * 3 * N1));
  CK(h, ensure(h->host_virial, sizeof(double) * 9 * S));
  rc = soapgap_compute(h, batch, SOAPGAP_ENERGY | SOAPGAP_FORCES | SOAPGAP_VIRIAL, nullptr, nullptr,
                       nullptr, (double*)h->host_e_struct.p, (double*)h->host_forces.p,
                       (double*)h->host_virial.p, stream);
  if (rc != SOAPGAP_OK) return rc;
  soapgap_handle::TilePlan best{};
  if (N > 0) {
    // the neighbour sweep (both paths): per bin or per atom, timed over whole evaluations
    // (the list is rebuilt at every call without a skin; with one, the sweep only runs on
    // rebuilds and the default is kept)
    const long long key = plan_key(h, N, h->last_pairs);
    float best_nb = -1.f;
    for (int v = 1; v <= 2 && h->skin == 0.0; ++v) {
      h->plans[key].nbr_sweep = v;
      double t = 0.0;
      for (int rep = 0; rep < 3; ++rep) {
        rc = soapgap_compute(h, batch, SOAPGAP_ENERGY | SOAPGAP_TIMING, nullptr, nullptr, nullptr,
                             (double*)h->host_e_struct.p, nullptr, nullptr, stream);
        if (rc != SOAPGAP_OK) return rc;
        double ms[SOAPGAP_N_STAGES] = {};
        rc = soapgap_stage_times(h, ms);
        if (rc != SOAPGAP_OK) return rc;
        if (rep > 0) t += ms[0];
      }
      if (best_nb < 0.f || t < best_nb) {
        best_nb = (float)t;
        best.nbr_sweep = v;
      }
    }
    h->plans[key].nbr_sweep = best.nbr_sweep;
    rc = soapgap_compute(h, batch, SOAPGAP_ENERGY | SOAPGAP_FORCES | SOAPGAP_VIRIAL, nullptr, nullptr,
                         nullptr, (double*)h->host_e_struct.p, (double*)h->host_forces.p,
                         (double*)h->host_virial.p, stream);
    if (rc != SOAPGAP_OK) return rc;
  }
  if (h->mixed && N > 0) {
    // each stage is idempotent on the handle's state after that evaluation: time its
    // candidates one after the other, keeping the others' choices fixed
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    float best_ms = -1.f;
    // the forward pair kernel: FP32 FMA or tensor-core contraction; afterwards the variant
    // of the evaluation above runs again, so that c matches the stages computed from it
    {
      const FwdArgs<float> fa = fwd_args<float>(h, N, batch->species);
      const int used = plan_for(h, N).pair_fwd;
      for (int v = 1; v <= 2; ++v) {
        if (v == 2 && !sg_pair_forward_mma_supported(h->cls)) continue;
        float ms = 0.f;
        TL(time_launches(h, st, e0, e1, 2, [&] { return launch_forward<float>(h, fa, v, st); }, &ms));
        if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
          best.pair_fwd = v;
          best_ms = ms;
        }
      }
      CK(h, launch_forward<float>(h, fa, used, st));
    }
    best_ms = -1.f;
    for (int w = 2; w <= SG_ADJ_TCGEN05; ++w) {
      AdjArgs<float> aa = adj_args<float>(h, N, batch->species);
      if (w == SG_ADJ_TCGEN05 && !sg_pair_adjoint_tc_supported(aa, h->cls)) continue;
      aa.warps = w;
      float ms = 0.f;
      TL(time_launches(h, st, e0, e1, 2, [&] { return sg_pair_adjoint<float>(aa, h->cls, true, st); }, &ms));
      if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
        best.adj_warps = w;
        best_ms = ms;
      }
    }
    // the GAP forward (its partial sums and kernel derivatives), then the backward on them
    GapTcModel tm = h->tcm;
    best_ms = -1.f;
    for (int c = 0; c < SG_GAP_FWD_CFGS; ++c) {
      tm.fwd_cfg = c;
      float ms = 0.f;
      TL(time_launches(h, st, e0, e1, 2, [&] {
        return sg_gap_tc_forward(tm, tm.terms, (const __half*)h->A16.p, (const float*)h->nrm.p,
                                 (const float*)h->uq.p, N, (float*)h->eps_part.p, (float*)h->r_part.p,
                                 (__half*)h->kp16.p, (int*)h->err.p, st);
      }, &ms));
      if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
        best.gap_fwd = c;
        best_ms = ms;
      }
    }
    tm.fwd_cfg = best.gap_fwd;
    CK(h, sg_gap_tc_forward(tm, tm.terms, (const __half*)h->A16.p, (const float*)h->nrm.p,
                            (const float*)h->uq.p, N, (float*)h->eps_part.p, (float*)h->r_part.p,
                            (__half*)h->kp16.p, (int*)h->err.p, st));
    best_ms = -1.f;
    for (int c = 0; c < SG_GAP_BWD_CFGS; ++c) {
      tm.bwd_cfg = c;
      float ms = 0.f;
      TL(time_launches(h, st, e0, e1, 2, [&] {
        return sg_gap_tc_backward(tm, (const __half*)h->kp16.p, (const float*)h->r_part.p, N, (float*)h->g.p,
                                  (int*)h->err.p, st);
      }, &ms));
      if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
        best.gap_bwd = c;
        best_ms = ms;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(h, cudaMemcpyAsync(h->h_err, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    if (*h->h_err) return fail(h, SOAPGAP_E_CUDA, device_error_text(*h->h_err));
    h->plans[plan_key(h, N, h->last_pairs)] = best;
  } else if (N > 0) {
    h->plans[plan_key(h, N, h->last_pairs)] = best;
    // the stages' outputs now come from the trial launches: a new evaluation is needed
    // before the adjoint's inputs are consistent again
    h->have_forward = false;
  }
  if (plan) {
    plan[0] = best.adj_warps;
    plan[1] = best.gap_fwd;
    plan[2] = best.gap_bwd;
    plan[3] = best.nbr_sweep;
    plan[4] = best.pair_fwd;
  }
  h->msg.clear();
  return SOAPGAP_OK;
}

// The batch's problem class as of its last evaluation on this handle.
static int plan_batch_key(soapgap_handle* h, const soapgap_batch* batch, long long* key) {
  int rc = check_batch(h, batch);
  if (rc != SOAPGAP_OK) return rc;
  if (!h->list_ok || h->list_atoms != batch->n_atoms)
    return fail(h, SOAPGAP_E_STATE, "plan: evaluate the batch synchronously first (its pair count sets its class)");
  *key = plan_key(h, batch->n_atoms, h->last_pairs);
  return SOAPGAP_OK;
}

extern "C" int soapgap_get_plan(soapgap_handle* h, const soapgap_batch* batch, int32_t* plan) {
  if (!h || !plan) return SOAPGAP_E_INVALID_ARG;
  long long key = 0;
  int rc = plan_batch_key(h, batch, &key);
  if (rc != SOAPGAP_OK) return rc;
  auto it = h->plans.find(key);
  const soapgap_handle::TilePlan p = it == h->plans.end() ? soapgap_handle::TilePlan{} : it->second;
  plan[0] = p.adj_warps;
  plan[1] = p.gap_fwd;
  plan[2] = p.gap_bwd;
  plan[3] = p.nbr_sweep;
  plan[4] = p.pair_fwd;
  h->msg.clear();
  return SOAPGAP_OK;
}

extern "C" int soapgap_set_plan(soapgap_handle* h, const soapgap_batch* batch, const int32_t* plan) {
  if (!h || !plan) return SOAPGAP_E_INVALID_ARG;
  if (!(plan[0] == 0 || (plan[0] >= 2 && plan[0] <= SG_ADJ_TCGEN05)) || plan[1] < 0 || plan[1] >= SG_GAP_FWD_CFGS ||
      plan[2] < 0 || plan[2] >= SG_GAP_BWD_CFGS || plan[3] < 0 || plan[3] > 2 || plan[4] < 0 || plan[4] > 2)
    return fail(h, SOAPGAP_E_INVALID_ARG,
                "set_plan: adjoint variant 0 or 2..5, GAP configurations, neighbour sweep and forward variant in range");
  long long key = 0;
  int rc = plan_batch_key(h, batch, &key);
  if (rc != SOAPGAP_OK) return rc;
  soapgap_handle::TilePlan p;
  p.adj_warps = plan[0];
  p.gap_fwd = plan[1];
  p.gap_bwd = plan[2];
  p.nbr_sweep = plan[3];
  p.pair_fwd = plan[4];
  h->plans[key] = p;
  h->have_forward = false;  // a new forward pass must produce the layout of the new plan
  h->msg.clear();
  return SOAPGAP_OK;
}

extern "C" int soapgap_set_gap_terms(soapgap_handle* h, int32_t terms) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  if (terms != 0 && terms != 1 && terms != 3)
    return fail(h, SOAPGAP_E_INVALID_ARG, "set_gap_terms: terms must be 0 (automatic), 1 or 3");
  h->gap_terms_forced = terms;
  if (h->has_model && h->mixed)
    h->tcm.terms = terms ? terms : (h->gap_probe_err >= 0 && h->gap_probe_err <= 1e-5 ? 1 : 3);
  h->msg.clear();
  return SOAPGAP_OK;
}

extern "C" int soapgap_gap_terms(const soapgap_handle* h, int32_t* terms, double* probe_err) {
  if (!h || !terms) return SOAPGAP_E_INVALID_ARG;
  *terms = (h->has_model && h->mixed) ? h->tcm.terms : 0;
  if (probe_err) *probe_err = (h->has_model && h->mixed) ? h->gap_probe_err : -1.0;
  return SOAPGAP_OK;
}

extern "C" int soapgap_set_skin(soapgap_handle* h, double skin) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  if (!(skin >= 0.0) || !std::isfinite(skin)) return fail(h, SOAPGAP_E_INVALID_ARG, "skin must be >= 0");
  h->skin = skin;
  h->ref_valid = false;  // the next call rebuilds with the new list radius
  h->msg.clear();
  return SOAPGAP_OK;
}

extern "C" int soapgap_last_rebuild(const soapgap_handle* h, int32_t* rebuilt) {
  if (!h || !rebuilt) return SOAPGAP_E_INVALID_ARG;
  *rebuilt = h->last_rebuild;
  return SOAPGAP_OK;
}

extern "C" int soapgap_verlet(soapgap_handle* h, const soapgap_batch* batch, double* pos, double* vel,
                              const double* forces, const double* inv_mass, double dt, int32_t drift,
                              void* stream) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  int rc = check_batch(h, batch);
  if (rc != SOAPGAP_OK) return rc;
  if (!pos || !vel || !forces || !inv_mass || !std::isfinite(dt))
    return fail(h, SOAPGAP_E_INVALID_ARG, "verlet needs pos, vel, forces, inv_mass and a finite dt");
  CK(h, sg_verlet(batch->n_atoms, pos, vel, forces, inv_mass, dt, drift != 0, (cudaStream_t)stream));
  h->msg.clear();
  return SOAPGAP_OK;
}

// ---------------------------------------------------------------- fitting-matrix rows
static void dmark(soapgap_handle* h, int slot, cudaStream_t st) {
  if (h->dev_timed) cudaEventRecord(h->dev_ev[slot], st);
}

template <typename T>
static int design(soapgap_handle* h, const soapgap_batch* b, uint32_t flags, void* k_atom, double* k_struct,
                  void* dk, cudaStream_t st) {
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  const size_t es = sizeof(T);
  dmark(h, 0, st);
  int rc = run<T>(h, b, SOAPGAP_DESC, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                  false, st);
  if (rc != SOAPGAP_OK) return rc;
  h->dstage_ran[0] = true;
  const int N = b->n_atoms, S = b->n_struct, M = h->M, D = h->D;
  const bool want_k = (flags & SOAPGAP_DESIGN_K) != 0, want_ks = (flags & SOAPGAP_DESIGN_KSTRUCT) != 0;
  const bool want_dk = (flags & SOAPGAP_DESIGN_DK) != 0;
  dmark(h, 1, st);
  if (want_ks) CK(h, cudaMemsetAsync(k_struct, 0, sizeof(double) * (size_t)S * M, st));
  if (want_dk && N > 0) CK(h, cudaMemsetAsync(dk, 0, es * (size_t)N * 3 * M, st));
  const size_t N1 = (size_t)std::max(N, 1);
  const int ldw = h->mixed ? h->tcm.mp : M;
  T* kbuf = (T*)k_atom;
  if (!want_k) {
    ENS(h, h->dk_k, es * N1 * M);
    kbuf = (T*)h->dk_k.p;
  }
  T2* wv = nullptr;
  if (want_dk) {
    ENS(h, h->dk_wv, sizeof(T2) * N1 * ldw);
    wv = (T2*)h->dk_wv.p;
  }
  if (N > 0 && (want_k || want_ks || want_dk)) {
    h->dstage_ran[1] = true;
    if constexpr (sizeof(T) == 4) {
      const GapTcModel& tm = h->tcm;
      ENS(h, h->A16, sizeof(__half) * N1 * 3 * tm.dp);
      ENS(h, h->nrm, sizeof(float) * N1);
      ENS(h, h->uq, sizeof(float) * N1);
      CK(h, sg_gap_tc_prepare((const float*)h->q.p, N, D, tm.dp, tm.qbar, (__half*)h->A16.p, (float*)h->nrm.p,
                              (float*)h->uq.p, 3, st));
      CK(h, sg_tc_kernel_rows(tm, (const __half*)h->A16.p, (const float*)h->nrm.p, (const float*)h->uq.p, N, M,
                              (const float*)h->pnorm.p, kbuf, wv, (int*)h->err.p, st));
    } else {
      CK(h, sg_kernel_rows_f64((const double*)h->q.p, N, (const double*)h->qs.p, M, D, h->zeta,
                               (const double*)h->pnorm.p, kbuf, wv, ldw, st));
    }
    if (want_ks) CK(h, sg_struct_rows<T>(kbuf, N, M, (const int*)h->atom_struct.p, k_struct, st));
  }
  dmark(h, 2, st);
  if (want_dk && N > 0) {
    h->dstage_ran[2] = h->dstage_ran[3] = true;
    const long long P = h->last_pairs;
    const long long ncols = 3 * (P + N);
    if (ncols > 0x7fffffffLL - 256)
      return fail(h, SOAPGAP_E_UNSUPPORTED, "too many Jacobian columns (3 (pairs + atoms) >= 2^31): split the batch");
    const int ld = h->mixed ? h->tcm.dpd : D;
    {
      // the table path writes only the first D + 2 entries of each column: the padding up to
      // ld stays as zeroed at allocation (the sparse operand is zero there too)
      const size_t cap_before = h->dk_J.cap;
      ENS(h, h->dk_J, (size_t)ncols * ld * (h->mixed ? sizeof(__half) : sizeof(double)));
      if (h->dk_J.cap != cap_before) CK(h, cudaMemsetAsync(h->dk_J.p, 0, h->dk_J.cap, st));
    }
    ENS(h, h->dk_at, sizeof(int2) * (size_t)ncols);
    ENS(h, h->dk_v, sizeof(Vec4<T>) * (size_t)ncols);
    JacArgs<T> ja{};
    ja.n_atoms = N;
    ja.nsp = h->prm.n_species;
    ja.nmax = h->prm.n_max;
    ja.lmax = h->prm.l_max;
    ja.dim = D;
    ja.ld = ld;
    ja.seg_offs = (const int*)h->seg_offs.p;
    ja.rev = (const int*)h->rev.p;
    ja.pair_j = (const int*)h->pair_j.p;
    ja.pair_r = (const Vec4<T>*)h->pair_r.p;
    ja.table = (const float*)h->table.p;
    ja.ti = h->ti;
    ja.p = h->dp;
    if constexpr (sizeof(T) == 4) {
      ja.yc = h->yc32;
      ja.bc = h->bc32;
      ja.qbar = h->tcm.qbar;
    } else {
      ja.yc = h->yc64;
      ja.bc = h->bc64;
      ja.qbar = nullptr;
    }
    ja.c = (const T*)h->c.p;
    ja.q = (const T*)h->q.p;
    ja.J = h->dk_J.p;
    ja.col_at = (int2*)h->dk_at.p;
    ja.col_v = (Vec4<T>*)h->dk_v.p;
    cudaError_t e = sg_design_jacobian<T>(ja, h->cls, h->mixed, st);
    if (e == cudaErrorInvalidConfiguration)
      return fail(h, SOAPGAP_E_UNSUPPORTED, "descriptor too large for the Jacobian kernel's shared memory");
    CK(h, e);
    dmark(h, 3, st);
    if constexpr (sizeof(T) == 4)
      CK(h, sg_tc_design_grad(h->tcm, M, (const __half*)h->dk_J.p, ncols, (const int2*)h->dk_at.p,
                              (const float4*)h->dk_v.p, wv, (float*)dk, (int*)h->err.p, st));
    else
      CK(h, sg_design_grad_f64((const double*)h->qs.p, M, D, (const double*)h->dk_J.p, ncols,
                               (const int2*)h->dk_at.p, (const Vec4<double>*)h->dk_v.p, wv, ldw, (double*)dk, st));
  } else {
    dmark(h, 3, st);
  }
  dmark(h, 4, st);
  CK(h, cudaMemcpyAsync(h->h_err, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if (*h->h_err) return fail(h, SOAPGAP_E_INVALID_ARG, device_error_text(*h->h_err));
  h->msg.clear();
  return SOAPGAP_OK;
}

extern "C" int soapgap_design(soapgap_handle* h, const soapgap_batch* batch, uint32_t flags, void* k_atom,
                              double* k_struct, void* dk, void* stream) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  int rc = check_batch(h, batch);
  if (rc != SOAPGAP_OK) return rc;
  if (flags & ~(SOAPGAP_DESIGN_K | SOAPGAP_DESIGN_KSTRUCT | SOAPGAP_DESIGN_DK | SOAPGAP_TIMING))
    return fail(h, SOAPGAP_E_INVALID_ARG, "unknown flag bits for soapgap_design");
  if (!h->has_model) return fail(h, SOAPGAP_E_STATE, "no sparse set: call soapgap_set_model first");
  if ((flags & SOAPGAP_DESIGN_K) && !k_atom) return fail(h, SOAPGAP_E_INVALID_ARG, "DESIGN_K needs k_atom");
  if ((flags & SOAPGAP_DESIGN_KSTRUCT) && !k_struct)
    return fail(h, SOAPGAP_E_INVALID_ARG, "DESIGN_KSTRUCT needs k_struct");
  if ((flags & SOAPGAP_DESIGN_DK) && !dk) return fail(h, SOAPGAP_E_INVALID_ARG, "DESIGN_DK needs dk");
  h->async_call = false;
  h->timed = false;
  h->dev_timed = (flags & SOAPGAP_TIMING) != 0;
  for (int k = 0; k < SOAPGAP_N_DESIGN_STAGES; ++k) h->dstage_ran[k] = false;
  if (h->dev_timed && !h->dev_made) {
    for (int k = 0; k <= SOAPGAP_N_DESIGN_STAGES; ++k) CK(h, cudaEventCreate(&h->dev_ev[k]));
    h->dev_made = true;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (h->mixed) return design<float>(h, batch, flags, k_atom, k_struct, dk, st);
  return design<double>(h, batch, flags, k_atom, k_struct, dk, st);
}

extern "C" int soapgap_design_times(const soapgap_handle* h, double* ms) {
  if (!h || !ms) return SOAPGAP_E_INVALID_ARG;
  if (!h->dev_timed || !h->dev_made) return SOAPGAP_E_STATE;
  for (int k = 0; k < SOAPGAP_N_DESIGN_STAGES; ++k) {
    float t = 0.f;
    ms[k] = 0.0;
    if (h->dstage_ran[k] && cudaEventElapsedTime(&t, h->dev_ev[k], h->dev_ev[k + 1]) == cudaSuccess) ms[k] = t;
  }
  return SOAPGAP_OK;
}

extern "C" int soapgap_kernel_rows(soapgap_handle* h, const void* q, int32_t n, void* k, void* stream) {
  if (!h) return SOAPGAP_E_INVALID_ARG;
  if (!h->has_model) return fail(h, SOAPGAP_E_STATE, "no sparse set: call soapgap_set_model first");
  if (n < 0 || (n > 0 && (!q || !k))) return fail(h, SOAPGAP_E_INVALID_ARG, "kernel_rows needs q, k and n >= 0");
  if (n == 0) return SOAPGAP_OK;
  h->async_call = false;
  cudaStream_t st = (cudaStream_t)stream;
  CK(h, cudaMemsetAsync(h->err.p, 0, sizeof(int), st));
  if (h->mixed) {
    const GapTcModel& tm = h->tcm;
    CK(h, ensure(h->A16, sizeof(__half) * (size_t)n * 3 * tm.dp));
    CK(h, ensure(h->nrm, sizeof(float) * (size_t)n));
    CK(h, ensure(h->uq, sizeof(float) * (size_t)n));
    CK(h, sg_gap_tc_prepare((const float*)q, n, h->D, tm.dp, tm.qbar, (__half*)h->A16.p, (float*)h->nrm.p,
                            (float*)h->uq.p, 3, st));
    CK(h, sg_tc_kernel_rows(tm, (const __half*)h->A16.p, (const float*)h->nrm.p, (const float*)h->uq.p, n, h->M,
                            nullptr, (float*)k, nullptr, (int*)h->err.p, st));
  } else {
    CK(h, sg_kernel_rows_f64((const double*)q, n, (const double*)h->qs.p, h->M, h->D, h->zeta, nullptr,
                             (double*)k, nullptr, 0, st));
  }
  CK(h, cudaMemcpyAsync(h->h_err, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if (*h->h_err) return fail(h, SOAPGAP_E_CUDA, device_error_text(*h->h_err));
  h->msg.clear();
  return SOAPGAP_OK;
}
