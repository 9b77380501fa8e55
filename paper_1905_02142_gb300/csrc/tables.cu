// Radial table of the mixed-precision path and the central-atom constants.
//
// Every quantity of a neighbour that depends on its distance only -- the orthonormal-
// basis radial coefficients b_n(r) (Eq. 01 with W = S^-1/2, Sec. III.A) and the angular
// factors 4 pi ilexp(x; l) (Sec. III.C) -- is evaluated here in FP64 with the paper's
// recursion (Eq. 04 and its erf seed, Gaussian-product buffer of Sec. III.B, closed-form
// Gaussian row) at the nodes r_k = k h, together with d/dr by forward-mode dual numbers.
// The FP32 pair kernels interpolate these nodes (cubic Hermite) instead of running the
// recursion per pair: in FP32 the per-pair primitive-basis coefficients lose their
// accuracy in W (cond(S) grows like a Hilbert matrix), which the FP64 nodes avoid.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "soapmath.cuh"
#include "table.cuh"

template <int NC, int LC>
__global__ void table_kernel(DevParams p, BasisConst<double> bc, TableInfo ti, float* table) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > ti.K) return;
  const double r = (k == ti.K) ? p.rc : k * ti.h;
  using D = Dual<double>;
  D rd(r, 1.0);
  D ba[NC];
  radial_alpha<D, NC>(rd, p, ba);
  D sp = p.s0p + p.ap * rd;
  D z = rd * rd / (sp * sp);
  D il[LC + 1];
  ilexp_all<D, LC>(z, il);
  float* v = table + (size_t)k * 2 * ti.fp;
  float* dv = v + ti.fp;
  for (int j = 0; j < ti.fp; ++j) { v[j] = 0.f; dv[j] = 0.f; }
  for (int n = 0; n < p.nmax; ++n) {
    D acc(0.0);
    for (int a = 0; a < p.nmax; ++a) acc = acc + bc.W[n][a] * ba[a];
    v[n] = (float)acc.v;
    dv[n] = (float)(ti.h * acc.d);
  }
  const double FOUR_PI = 12.566370614359172;
  for (int l = 0; l <= p.lmax; ++l) {
    double w = FOUR_PI * (p.eq08 ? (2.0 * l + 1.0) : 1.0);
    v[TableDims<NC, LC>::NCP + l] = (float)(w * il[l].v);
    dv[TableDims<NC, LC>::NCP + l] = (float)(ti.h * w * il[l].d);
  }
}

cudaError_t sg_build_table(const DevParams& p, const BasisConst<double>& W, int cls,
                           const TableInfo& ti, float* table, cudaStream_t st) {
  const int threads = 64, blocks = (ti.K + 1 + threads - 1) / threads;
  switch (cls) {
    case 0: table_kernel<6, 6><<<blocks, threads, 0, st>>>(p, W, ti, table); break;
    case 1: table_kernel<8, 8><<<blocks, threads, 0, st>>>(p, W, ti, table); break;
    case 2: table_kernel<10, 10><<<blocks, threads, 0, st>>>(p, W, ti, table); break;
    default: table_kernel<12, 12><<<blocks, threads, 0, st>>>(p, W, ti, table); break;
  }
  ++sg_kernel_launches;
  return cudaGetLastError();
}

// central atom (r = 0): ilexp(0; l) = delta_l0 and Y_00 = 1/sqrt(4 pi), so it adds
// central_weight * sqrt(4 pi) * b(0) to the l = 0 coefficients of its own species.
__global__ void central_kernel(DevParams p, BasisConst<double> bc, double* out_n,
                               double* out_alpha) {
  double ba[SG_MAX_NMAX];
  radial_alpha<double, SG_MAX_NMAX>(0.0, p, ba);
  const double s = p.cw * 3.5449077018110318;  // sqrt(4 pi)
  for (int a = 0; a < p.nmax; ++a) out_alpha[a] = s * ba[a];
  for (int n = 0; n < p.nmax; ++n) {
    double acc = 0.0;
    for (int a = 0; a < p.nmax; ++a) acc += bc.W[n][a] * ba[a];
    out_n[n] = s * acc;
  }
}

cudaError_t sg_central_terms(const DevParams& p, const BasisConst<double>& W, double* out_n,
                             double* out_alpha, cudaStream_t st) {
  central_kernel<<<1, 1, 0, st>>>(p, W, out_n, out_alpha);
  ++sg_kernel_launches;
  return cudaGetLastError();
}

// Powers of two that bring the tensor-core forward's FP16 operands near 2^13 (FP16 holds up
// to 65504 and is normal from 2^-14): sb for b_n, sa for a_lm = 4 pi ilexp_l Y_lm, from
// the table's node values (Hermite overshoot between nodes stays well inside the margin)
// and |Y_lm| <= sqrt((2l + 1) / 4 pi) for orthonormal real harmonics.  Reads the table
// back to the host (set-up only).
cudaError_t sg_fwd_mma_scales(const float* table, const TableInfo& ti, int ncp, int nmax, int lmax, float* sa,
                              float* sb) {
  std::vector<float> h((size_t)(ti.K + 1) * 2 * ti.fp);
  cudaError_t e = cudaMemcpy(h.data(), table, sizeof(float) * h.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  double bmax = 0.0, amax = 0.0;
  const double inv4pi = 1.0 / 12.566370614359172;
  for (int k = 0; k <= ti.K; ++k) {
    const float* v = h.data() + (size_t)k * 2 * ti.fp;  // values half-node
    for (int n = 0; n < nmax; ++n) bmax = std::max(bmax, (double)std::fabs(v[n]));
    for (int l = 0; l <= lmax; ++l)
      amax = std::max(amax, std::fabs((double)v[ncp + l]) * std::sqrt((2.0 * l + 1.0) * inv4pi));
  }
  auto scale = [](double m) {
    if (!(m > 0.0) || !std::isfinite(m)) return 1.f;
    int ex = 0;
    std::frexp(m, &ex);  // m < 2^ex
    ex = std::max(-100, std::min(100, ex));
    return std::ldexp(1.f, 13 - ex);
  };
  *sb = scale(bmax);
  *sa = scale(amax);
  return cudaSuccess;
}
