"""Radial basis of the new SOAP (Sec. III.A), oracle side.

phi_alpha(r) = (1 - r/r_cut)^(alpha+2) / N_alpha,  N_alpha = sqrt(r_cut / (2 alpha + 5)),
for alpha = 1 .. n_max-1, plus the auxiliary Gaussian of Eq. 06,
phi_nmax(r) = sqrt(2) / (sqrt(sigma_0r) pi^(1/4)) exp(-r^2 / (2 sigma_0r^2)).
The overlap matrix S_ab = int_0^r_cut phi_a phi_b dr is evaluated by quadrature of that
definition, and W = S^(-1/2) by a symmetric eigendecomposition (a library primitive), so
that g_n = sum_a W_na phi_a is orthonormal on [0, r_cut].  S is ill conditioned (cond(S)
~5e11 at n_max = 8, ~1e16 at n_max = 12, the paper's stated limit), so W is built with
40-digit mpmath arithmetic and only then rounded to FP64; in FP64 alone W would carry
relative errors near eps * cond(S).
"""
from __future__ import annotations

import functools
import math

import mpmath
import numpy as np


def poly_norm(alpha, r_cut: float):
    """N_alpha of Sec. III.A."""
    return np.sqrt(r_cut / (2.0 * np.asarray(alpha, dtype=np.float64) + 5.0))


def basis_functions(r: np.ndarray, n_max: int, r_cut: float, sigma_r0: float) -> np.ndarray:
    """[n_max, len(r)]: phi_1 .. phi_{n_max-1} (polynomials) and phi_{n_max} (Eq. 06)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty((n_max, r.size))
    t = 1.0 - r / r_cut
    for a in range(1, n_max):
        out[a - 1] = t ** (a + 2) / poly_norm(a, r_cut)
    out[n_max - 1] = (math.sqrt(2.0) / (math.sqrt(sigma_r0) * math.pi ** 0.25)
                      * np.exp(-r * r / (2.0 * sigma_r0 * sigma_r0)))
    return out


def gauss_legendre(a: float, b: float, panels: int = 64, order: int = 32):
    """Composite Gauss-Legendre nodes and weights on [a, b]."""
    x, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(a, b, panels + 1)
    nodes, weights = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        nodes.append(0.5 * (hi - lo) * x + 0.5 * (hi + lo))
        weights.append(0.5 * (hi - lo) * w)
    return np.concatenate(nodes), np.concatenate(weights)


def overlap_matrix(n_max: int, r_cut: float, sigma_r0: float) -> np.ndarray:
    """S_ab = int_0^r_cut phi_a(r) phi_b(r) dr (Sec. III.A), by quadrature."""
    r, w = gauss_legendre(0.0, r_cut)
    phi = basis_functions(r, n_max, r_cut, sigma_r0)
    return (phi * w[None, :]) @ phi.T


def overlap_matrix_mp(n_max: int, r_cut: float, sigma_r0: float, dps: int = 40):
    """S_ab (Sec. III.A) as an mpmath matrix, by Gauss-Legendre quadrature at ``dps`` digits."""
    with mpmath.workdps(dps):
        rc, s0 = mpmath.mpf(r_cut), mpmath.mpf(sigma_r0)
        gnorm = mpmath.sqrt(2) / (mpmath.sqrt(s0) * mpmath.pi ** mpmath.mpf(0.25))

        def phi(a, r):
            if a < n_max:
                return (1 - r / rc) ** (a + 2) / mpmath.sqrt(rc / (2 * a + 5))
            return gnorm * mpmath.exp(-r * r / (2 * s0 * s0))

        pts = mpmath.linspace(0, rc, 41)
        s = mpmath.matrix(n_max, n_max)
        for a in range(1, n_max + 1):
            for b in range(a, n_max + 1):
                v = mpmath.quad(lambda r: phi(a, r) * phi(b, r), pts, method="gauss-legendre")
                s[a - 1, b - 1] = v
                s[b - 1, a - 1] = v
        return s


@functools.lru_cache(maxsize=None)
def _orthonormaliser(n_max: int, r_cut: float, sigma_r0: float) -> np.ndarray:
    with mpmath.workdps(40):
        s = overlap_matrix_mp(n_max, r_cut, sigma_r0)
        ev, vec = mpmath.eigsy(s)
        if min(ev) <= 0:
            raise ValueError("overlap matrix is not positive definite")
        d = mpmath.diag([1 / mpmath.sqrt(e) for e in ev])
        w = vec * d * vec.T
        return np.array([[float(w[i, j]) for j in range(n_max)] for i in range(n_max)])


def orthonormaliser(n_max: int, r_cut: float, sigma_r0: float) -> np.ndarray:
    """W = S^(-1/2) (Sec. III.A), computed at 40 digits and rounded to FP64."""
    return _orthonormaliser(int(n_max), float(r_cut), float(sigma_r0)).copy()
