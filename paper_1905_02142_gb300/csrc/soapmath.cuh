// Per-pair mathematics of the separable-density SOAP (Caro 2019), written once as
// templates over the scalar type S: double, or Dual<double> to carry d/dr alongside the
// value (forward-mode differentiation for the radial derivatives of the adjoint).
#pragma once

#include <math.h>
#include "common.cuh"

// ---------------------------------------------------------------- dual numbers
template <typename T> struct Dual {
  T v, d;
  __host__ __device__ Dual() : v(0), d(0) {}
  __host__ __device__ Dual(T v_) : v(v_), d(0) {}
  __host__ __device__ Dual(T v_, T d_) : v(v_), d(d_) {}
};
template <typename T> __host__ __device__ inline Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <typename T> __host__ __device__ inline Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator+(T a, Dual<T> b) { return {a + b.v, b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator-(Dual<T> a, T b) { return {a.v - b, a.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator-(T a, Dual<T> b) { return {a - b.v, -b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <typename T> __host__ __device__ inline Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator/(Dual<T> a, T b) { return {a.v / b, a.d / b}; }
template <typename T> __host__ __device__ inline Dual<T> operator/(T a, Dual<T> b) {
  T q = a / b.v;
  return {q, -q * b.d / b.v};
}

__host__ __device__ inline double val(double x) { return x; }
__host__ __device__ inline double val(Dual<double> x) { return x.v; }

__host__ __device__ inline double s_exp(double x) { return exp(x); }
__host__ __device__ inline double s_expm1(double x) { return expm1(x); }
__host__ __device__ inline double s_erf(double x) { return erf(x); }
__host__ __device__ inline double s_erfc(double x) { return erfc(x); }
__host__ __device__ inline double s_sqrt(double x) { return sqrt(x); }
__host__ __device__ inline double s_pow(double x, double a) { return pow(x, a); }

#define SG_TWO_OVER_SQRTPI 1.1283791670955126
__host__ __device__ inline Dual<double> s_exp(Dual<double> x) { double e = exp(x.v); return {e, e * x.d}; }
__host__ __device__ inline Dual<double> s_expm1(Dual<double> x) { return {expm1(x.v), exp(x.v) * x.d}; }
__host__ __device__ inline Dual<double> s_erf(Dual<double> x) { return {erf(x.v), SG_TWO_OVER_SQRTPI * exp(-x.v * x.v) * x.d}; }
__host__ __device__ inline Dual<double> s_erfc(Dual<double> x) { return {erfc(x.v), -SG_TWO_OVER_SQRTPI * exp(-x.v * x.v) * x.d}; }
__host__ __device__ inline Dual<double> s_sqrt(Dual<double> x) { double s = sqrt(x.v); return {s, x.d / (2.0 * s)}; }
__host__ __device__ inline Dual<double> s_pow(Dual<double> x, double a) {
  double p = pow(x.v, a);
  // at x = 0 the slope is 0 for a > 1, x.d for a = 1; it is unbounded for a < 1 (the
  // amplitude polynomial only reaches 0 at r_cut, where no neighbour is kept)
  if (x.v == 0.0) return {p, a == 1.0 ? x.d : 0.0};
  return {p, a * pow(x.v, a - 1.0) * x.d};
}

// ------------------------------------------------------------- radial integrals
// erf(hi) - erf(lo), lo <= hi, through erfc when both arguments have the same sign.
template <typename S> __host__ __device__ inline S erf_difference(S lo, S hi) {
  if (val(lo) >= 0.0) return s_erfc(lo) - s_erfc(hi);
  if (val(hi) <= 0.0) return s_erfc(-hi) - s_erfc(-lo);
  return s_erf(hi) - s_erf(lo);
}

// J_k = int_a^b (1 - r/rc)^k exp(-(r - c)^2 / (2 w^2)) dr, k = 0..kmax (Sec. III.A):
// J_0 from erf (the b_{-2} seed), J_1 from J_0 (the b_{-3} term has a zero factor), then
// Eq. 04:  J_{k+2} = (k+1)(w/rc)^2 J_k + (1 - c/rc) J_{k+1}
//                    + (w^2/rc) [(1 - r/rc)^(k+1) exp(-(r-c)^2/(2w^2))]_a^b.
// Terms are added to J[] (callers zero it), scaled by `amp`.
template <typename S, int KMAX>
__host__ __device__ inline void radial_integrals_add(S c, S w, double a, double b, double rc,
                                                     S amp, S* J) {
  const double SQRT2 = 1.4142135623730951, SQRT_HALF_PI = 1.2533141373155003;
  S inv2w2 = 1.0 / (2.0 * w * w);
  S ga = s_exp(-(a - c) * (a - c) * inv2w2);
  S gb = s_exp(-(b - c) * (b - c) * inv2w2);
  S sw = SQRT2 * w;
  S jm2 = SQRT_HALF_PI * w * erf_difference((a - c) / sw, (b - c) / sw);
  S eps = (w * w) / (rc * rc);
  S beta = 1.0 - c / rc;
  S bcoef = (w * w) / rc;
  double ta = 1.0 - a / rc, tb = 1.0 - b / rc;
  S jm1 = beta * jm2 + bcoef * (gb - ga);
  J[0] = J[0] + amp * jm2;
  J[1] = J[1] + amp * jm1;
  double tak = ta, tbk = tb;
#pragma unroll
  for (int k = 0; k + 2 <= KMAX; ++k) {
    S jn = (double)(k + 1) * eps * jm2 + beta * jm1 + bcoef * (tbk * gb - tak * ga);
    J[k + 2] = J[k + 2] + amp * jn;
    jm2 = jm1;
    jm1 = jn;
    tak *= ta;
    tbk *= tb;
  }
}

// Overlap of the auxiliary Gaussian phi_nmax (Eq. 06) with the radial Gaussian on
// [0, inf): the closed form given after Eq. 04.
template <typename S> __host__ __device__ inline S gaussian_row(S r, S sr, double s0) {
  const double SQRT2 = 1.4142135623730951;
  S sstar = s_sqrt(s0 * s0 + sr * sr);
  double k = pow(3.141592653589793, 0.25) / sqrt(s0);
  return k * s_exp(-r * r / (2.0 * sstar * sstar)) * (s0 * sr / sstar) *
         (1.0 + s_erf(s0 * r / (SQRT2 * sr * sstar)));
}

// b_alpha (alpha = 1..nmax, primitive basis, including A_j of Eq. 15 and the density
// smoothing of Sec. III.B) for a neighbour at distance r.  NC >= nmax.
template <typename S, int NC>
__host__ __device__ inline void radial_alpha(S r, const DevParams& p, S* bout) {
  S sr = p.s0r + p.ar * r;
  S sp = p.s0p + p.ap * r;
  S x = r / p.rc;
  S poly = (1.0 - x) * (1.0 - x) * (1.0 + 2.0 * x);
  S damp = (p.amp_a == 0.0) ? S(1.0) : s_pow(poly, p.amp_a);
  S amp = damp / (sr * sp * sp);
  S J[NC + 2];
#pragma unroll
  for (int k = 0; k < NC + 2; ++k) J[k] = S(0.0);
  double rs = p.rs < p.rc ? p.rs : p.rc;
  radial_integrals_add<S, NC + 1>(r, sr, 0.0, rs, p.rc, S(1.0), J);
  if (rs < p.rc) {
    double tau = (p.rc - rs) / p.nf;
    S s2 = 1.0 / (1.0 / (sr * sr) + 1.0 / (tau * tau));
    S mu = s2 * (r / (sr * sr) + rs / (tau * tau));
    S cbuf = s_exp(-(r - rs) * (r - rs) / (2.0 * (sr * sr + tau * tau)));
    radial_integrals_add<S, NC + 1>(mu, s_sqrt(s2), rs, p.rc, p.rc, cbuf, J);
  }
  S grow = amp * gaussian_row(r, sr, p.s0r);
  // bout[a] = b_{alpha = a+1}: polynomials J_{alpha+2} / N_alpha, then the Gaussian row
#pragma unroll
  for (int a = 0; a < NC; ++a) {
    if (a + 3 <= NC + 1 && a + 1 < p.nmax)
      bout[a] = amp * J[a + 3] / sqrt(p.rc / (2.0 * (a + 1) + 5.0));
    else if (a + 1 == p.nmax)
      bout[a] = grow;
    else
      bout[a] = S(0.0);
  }
}

// ilexp(x; l) = e^{-z} i_l(z), z = x^2, for l = 0..LC (Sec. III.C).
//   z >= 30: the upward recursion of Sec. III.C from the closed forms for l = 0, 1
//            (well conditioned there: relative error < 1e-14 up to l = 13 in FP64);
//   0 < z < 30: the power series of i_l for the top two orders, then the recursion run
//            downwards (stable for the minimal solution i_l).
template <typename S, int LC> __host__ __device__ inline void ilexp_all(S z, S* il) {
  if (val(z) == 0.0) {
#pragma unroll
    for (int l = 0; l <= LC; ++l) il[l] = S(0.0);
    il[0] = 1.0 - z;  // exact value and slope at z = 0
    if (LC >= 1) il[1] = z / 3.0;
    return;
  }
  if (val(z) >= 30.0) {
    S e2 = s_exp(-2.0 * z);
    il[0] = -s_expm1(-2.0 * z) / (2.0 * z);
    if (LC >= 1) il[1] = ((z - 1.0) + e2 * (z + 1.0)) / (2.0 * z * z);
#pragma unroll
    for (int l = 2; l <= LC; ++l) il[l] = il[l - 2] - (double)(2 * l - 1) / z * il[l - 1];
    return;
  }
  const int LT = LC >= 1 ? LC : 1;
  S top[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int L = LT - t;
    double df = 1.0;
    for (int k = 2 * L + 1; k > 1; k -= 2) df *= k;
    S term = S(1.0 / df);
    for (int k = 0; k < L; ++k) term = term * z;
    S sum = term;
    S z2h = z * z * 0.5;
    for (int k = 0; k < 200; ++k) {
      term = term * z2h / (double)((k + 1) * (2 * L + 2 * k + 3));
      sum = sum + term;
      if (val(term) < 1e-18 * val(sum)) break;
    }
    top[t] = s_exp(-z) * sum;
  }
  S hi = top[0], lo = top[1];  // il[LT], il[LT-1]
  if (LT <= LC) il[LT] = hi;
  il[LT - 1] = lo;
#pragma unroll
  for (int l = LT - 1; l >= 1; --l) {
    S nx = hi + (double)(2 * l + 1) / z * lo;  // il[l-1]
    hi = lo;
    lo = nx;
    il[l - 1] = nx;
  }
}

// ------------------------------------------------------- real spherical harmonics
// Normalised real Y_lm on a unit vector u, pole-free Cartesian form:
//   Y_l0 = N~_l^0(z),  Y_{l,+m} = N~_l^m(z) Re(x+iy)^m,  Y_{l,-m} = N~_l^m(z) Im(x+iy)^m,
// N~_l^m the normalised d^m P_l/dz^m (sqrt(2) folded in for m > 0), by the recursion in l.
// The callback f(l, m, Y) receives every value, m-major order.
template <typename T, int LC, typename F>
__device__ __forceinline__ void for_each_ylm(T x, T y, T z, const YlmCoef<T>& yc, F&& f) {
  T cm = 1, sm = 0;
#pragma unroll
  for (int m = 0; m <= LC; ++m) {
    if (m > 0) {
      T c2 = x * cm - y * sm;
      sm = x * sm + y * cm;
      cm = c2;
    }
    T p2 = 0, p1 = yc.seed[m];
#pragma unroll
    for (int l = m; l <= LC; ++l) {
      T pl;
      if (l == m) pl = p1;
      else if (l == m + 1) pl = yc.s1[m] * z * p1;
      else pl = yc.a[l][m] * z * p1 - yc.b[l][m] * p2;
      if (l > m) { p2 = p1; p1 = pl; }
      if (m == 0) f(l, 0, pl);
      else { f(l, m, pl * cm); f(l, -m, pl * sm); }
    }
  }
}

// Same traversal with the gradient of the polynomial extension P_lm(x, y, z) with respect
// to u (its projection on the tangent plane, divided by r, is grad_r Y_lm(r_hat)).
// Column m of N~ and column m+1 (for dN~_l^m/dz) are both run as scalar recursions in l,
// so that with the loops unrolled every index is a compile-time constant.
template <typename T, int LC, typename F>
__device__ __forceinline__ void for_each_ylm_grad(T x, T y, T z, const YlmCoef<T>& yc, F&& f) {
  T cm = 1, sm = 0, cmm1 = 0, smm1 = 0;
#pragma unroll
  for (int m = 0; m <= LC; ++m) {
    if (m > 0) {
      const T c2 = x * cm - y * sm;
      const T s2 = x * sm + y * cm;
      cmm1 = cm;
      smm1 = sm;
      cm = c2;
      sm = s2;
    }
    T a2 = 0, a1 = yc.seed[m];                        // column m
    T b2 = 0, b1 = (m + 1 <= LC) ? yc.seed[m + 1] : T(0);  // column m+1
#pragma unroll
    for (int l = m; l <= LC; ++l) {
      T pl;
      if (l == m) {
        pl = a1;
      } else {
        pl = (l == m + 1) ? yc.s1[m] * z * a1 : yc.a[l][m] * z * a1 - yc.b[l][m] * a2;
        a2 = a1;
        a1 = pl;
      }
      T ql = T(0);
      if (m + 1 <= LC && l >= m + 1) {
        if (l == m + 1) {
          ql = b1;
        } else {
          ql = (l == m + 2) ? yc.s1[m + 1] * z * b1 : yc.a[l][m + 1] * z * b1 - yc.b[l][m + 1] * b2;
          b2 = b1;
          b1 = ql;
        }
      }
      const T dz = yc.d[l][m] * ql;  // dN~_l^m/dz
      if (m == 0) {
        f(l, 0, pl, T(0), T(0), dz);
      } else {
        const T fm = (T)m * pl;
        f(l, m, pl * cm, fm * cmm1, -fm * smm1, dz * cm);
        f(l, -m, pl * sm, fm * smm1, fm * cmm1, dz * sm);
      }
    }
  }
}

// Coefficients of the normalised real-harmonic recursion, staged in shared memory so that
// (l, m) loops can run rolled (small code, no instruction-cache pressure).  Column
// SG_MAX_LMAX + 1 is zero (the seed of the column past the last).
template <typename T> struct YlmShared {
  T seed[SG_MAX_LMAX + 2], s1[SG_MAX_LMAX + 2];
  T a[SG_MAX_LMAX + 1][SG_MAX_LMAX + 2], b[SG_MAX_LMAX + 1][SG_MAX_LMAX + 2];
  T d[SG_MAX_LMAX + 1][SG_MAX_LMAX + 2];
};

// Block-cooperative copy of the recursion coefficients into shared memory.
template <typename T>
__device__ inline void load_ylm_shared(YlmShared<T>& ys, const YlmCoef<T>& yc) {
  for (int k = threadIdx.x; k <= SG_MAX_LMAX; k += blockDim.x) {
    ys.seed[k] = yc.seed[k];
    ys.s1[k] = yc.s1[k];
  }
  if (threadIdx.x == 0) {
    ys.seed[SG_MAX_LMAX + 1] = T(0);
    ys.s1[SG_MAX_LMAX + 1] = T(0);
  }
  for (int k = threadIdx.x; k < (SG_MAX_LMAX + 1) * (SG_MAX_LMAX + 2); k += blockDim.x) {
    const int l = k / (SG_MAX_LMAX + 2), m = k - l * (SG_MAX_LMAX + 2);
    ys.a[l][m] = m <= SG_MAX_LMAX ? yc.a[l][m] : T(0);
    ys.b[l][m] = m <= SG_MAX_LMAX ? yc.b[l][m] : T(0);
    ys.d[l][m] = m <= SG_MAX_LMAX ? yc.d[l][m] : T(0);
  }
}
