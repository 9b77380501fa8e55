// Orthonormaliser W = S^-1/2 of the radial basis (Sec. III.A), computed on the host in
// IEEE binary128 and rounded to FP64.
//
// S (the overlap matrix of the n_max-1 polynomials (1 - r/rc)^(alpha+2)/N_alpha and the
// auxiliary Gaussian of Eq. 06) is ill conditioned: cond(S) grows like a Hilbert matrix,
// ~5e11 at n_max = 8 and ~1e16 at n_max = 12, which is why the paper limits n_max to 12.
// An eigendecomposition in FP64 would leave W with relative errors near eps*cond(S), so
// S and its eigendecomposition are carried in binary128 (compiled by the host compiler;
// glibc provides the _Float128 math functions on x86-64 and AArch64).
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include <math.h>

#include <vector>

typedef _Float128 Q;

static Q qN(int a, Q rc) { return sqrtf128(rc / (Q)(2 * a + 5)); }

// J_k = int_0^rc (1 - r/rc)^k exp(-r^2 / (2 w^2)) dr through the recursion of Eq. 04
// (centre c = 0), started from the erf seed.
static void j_integrals(Q rc, Q w, int kmax, Q* J) {
  const Q pi = 4 * atanf128((Q)1);
  const Q sqrt2 = sqrtf128((Q)2);
  const Q gb = expf128(-rc * rc / (2 * w * w));
  const Q ga = 1;
  J[0] = w * sqrtf128(pi / 2) * erff128(rc / (sqrt2 * w));
  const Q eps = (w * w) / (rc * rc), beta = 1, bcoef = (w * w) / rc;
  J[1] = beta * J[0] + bcoef * (gb - ga);
  // boundary factors: (1 - r/rc)^(k+1) is 1 at r = 0 and 0 at r = rc
  for (int k = 0; k + 2 <= kmax; ++k) J[k + 2] = (Q)(k + 1) * eps * J[k] + beta * J[k + 1] + bcoef * (0 - ga);
}

static void jacobi(int n, std::vector<Q>& a, std::vector<Q>& ev, std::vector<Q>& v) {
  v.assign(n * n, 0);
  for (int i = 0; i < n; ++i) v[i * n + i] = 1;
  for (int sweep = 0; sweep < 200; ++sweep) {
    Q off = 0, diag = 0;
    for (int p = 0; p < n; ++p) {
      diag += a[p * n + p] * a[p * n + p];
      for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
    }
    if (off <= (Q)1e-70 * diag) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const Q apq = a[p * n + q];
        if (apq == 0) continue;
        const Q theta = (a[q * n + q] - a[p * n + p]) / (2 * apq);
        const Q t = (theta >= 0 ? (Q)1 : (Q)-1) / (fabsf128(theta) + sqrtf128(theta * theta + 1));
        const Q c = 1 / sqrtf128(t * t + 1), s = t * c;
        for (int k = 0; k < n; ++k) {
          const Q akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const Q apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const Q vkp = v[k * n + p], vkq = v[k * n + q];
          v[k * n + p] = c * vkp - s * vkq;
          v[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
}

// Writes W (row-major n_max x n_max, FP64) and cond(S); returns 0, or -1 if S is not
// positive definite even in binary128.
int sg_orthonormaliser_q(int nmax, double rc_d, double s0_d, double* W, double* cond) {
  const Q rc = rc_d, s0 = s0_d;
  const Q pi = 4 * atanf128((Q)1);
  std::vector<Q> S(nmax * nmax, 0);
  for (int a = 1; a < nmax; ++a)
    for (int b = 1; b < nmax; ++b)
      S[(a - 1) * nmax + (b - 1)] = rc / ((Q)(a + b + 5) * qN(a, rc) * qN(b, rc));
  std::vector<Q> J(nmax + 3, 0);
  j_integrals(rc, s0, nmax + 2, J.data());
  const Q gnorm = sqrtf128((Q)2) / (sqrtf128(s0) * sqrtf128(sqrtf128(pi)));
  for (int a = 1; a < nmax; ++a) {
    const Q v = gnorm * J[a + 2] / qN(a, rc);
    S[(a - 1) * nmax + nmax - 1] = v;
    S[(nmax - 1) * nmax + a - 1] = v;
  }
  S[nmax * nmax - 1] = erff128(rc / s0);
  std::vector<Q> ev, V;
  jacobi(nmax, S, ev, V);
  Q emin = ev[0], emax = ev[0];
  for (Q e : ev) {
    if (e < emin) emin = e;
    if (e > emax) emax = e;
  }
  if (!(emin > 0)) return -1;
  *cond = (double)(emax / emin);
  for (int a = 0; a < nmax; ++a)
    for (int b = 0; b < nmax; ++b) {
      Q w = 0;
      for (int k = 0; k < nmax; ++k) w += V[a * nmax + k] * V[b * nmax + k] / sqrtf128(ev[k]);
      W[a * nmax + b] = (double)w;
    }
  return 0;
}
