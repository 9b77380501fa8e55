"""Pins of the oracle's radial basis and radial coefficients (Sec. III.A, III.B, Eq. 15).

Each check compares the oracle with something other than itself: closed-form
integrals, direct numerical quadrature of the defining integrals, or values printed
in the paper.
"""
import math

import numpy as np
import pytest
import torch

from oracle import Params, basis, soap

DT = torch.float64


def quad(f, a, b, panels=400, order=24):
    r, w = basis.gauss_legendre(a, b, panels=panels, order=order)
    return np.sum(w * f(r))


@pytest.mark.parametrize("n_max,r_cut", [(4, 3.7), (8, 5.0), (12, 4.5)])
def test_polynomial_overlaps_closed_form(n_max, r_cut):
    # Sec. III.A: int_0^rc (1-r/rc)^(a+b+4) dr = rc/(a+b+5), and N_a normalises phi_a
    s = basis.overlap_matrix(n_max, r_cut, 0.5)
    for a in range(1, n_max):
        for b in range(1, n_max):
            exact = r_cut / ((a + b + 5) * basis.poly_norm(a, r_cut) * basis.poly_norm(b, r_cut))
            assert abs(s[a - 1, b - 1] - exact) < 1e-13
        assert abs(s[a - 1, a - 1] - 1.0) < 1e-13


@pytest.mark.parametrize("sigma", [0.12, 0.5])
def test_gaussian_basis_function_normalised(sigma):
    # Eq. 06 is normalised on [0, inf); on [0, rc] the deficit is erfc(rc/sigma)
    s = basis.overlap_matrix(6, 5.0, sigma)
    assert abs(s[-1, -1] - math.erf(5.0 / sigma)) < 1e-13


@pytest.mark.parametrize("n_max", [3, 4, 6])
def test_orthonormal_basis_by_quadrature(n_max):
    # g_n = sum_a W_na phi_a must be orthonormal on [0, rc] (Sec. III.A)
    r_cut, sig = 4.0, 0.5
    w = basis.orthonormaliser(n_max, r_cut, sig)
    r, wq = basis.gauss_legendre(0.0, r_cut, panels=300, order=20)
    g = w @ basis.basis_functions(r, n_max, r_cut, sig)
    gram = (g * wq[None, :]) @ g.T
    cond = np.linalg.cond(basis.overlap_matrix(n_max, r_cut, sig))
    assert np.abs(gram - np.eye(n_max)).max() < 1e3 * 2.2e-16 * cond


def test_overlap_matrix_degenerates_beyond_nmax_12(golden):
    # Sec. III.A: linear dependencies make the basis unusable for n_max > 12
    lim = golden["overlap_singularity"]["n_max_limit"]
    ev_ok = np.linalg.eigvalsh(basis.overlap_matrix(4, 5.0, 0.5))
    ev_bad = np.linalg.eigvalsh(basis.overlap_matrix(lim + 2, 5.0, 0.5))
    assert ev_ok.min() / ev_ok.max() > 1e-8
    assert ev_bad.min() / ev_bad.max() < 1e-15


def test_smoothing_value_at_hard_cutoff(golden):
    g = golden["smoothing_at_hard_cutoff"]
    for rs, rh in [(4.5, 5.0), (2.0, 3.7), (3.0, 6.0)]:
        P = Params(r_cut=rh, r_soft=rs, sigma_r0=0.5, sigma_p0=0.5, n_f=g["n_f"])
        f = float(soap.smoothing_function(torch.tensor([rh - 1e-12], dtype=DT), P))
        assert f == pytest.approx(g["value"], rel=10 ** (-g["printed_digits"]) * 2)
        assert abs(f - math.exp(-g["n_f"] ** 2 / 2)) < 1e-10
        assert float(soap.smoothing_function(torch.tensor([rs - 1e-9], dtype=DT), P)) == 1.0
        assert float(soap.smoothing_function(torch.tensor([rh + 1e-9], dtype=DT), P)) == 0.0


CASES = [(c, w) for c in (0.0, 0.3, 1.7, 3.9, 4.6, 4.95) for w in (0.12, 0.2, 0.5)]


@pytest.mark.parametrize("c,w", CASES)
@pytest.mark.parametrize("a,b", [(0.0, 4.5), (4.5, 5.0), (0.0, 5.0)])
def test_recursion_matches_quadrature(c, w, a, b):
    # Eq. 04 with the erf seed, against direct quadrature of the defining integral
    rc, kmax = 5.0, 14
    jr = soap.radial_integrals(torch.tensor([c], dtype=DT), torch.tensor([w], dtype=DT),
                               a, b, rc, kmax)[0].numpy()
    jq = np.array([quad(lambda r: (1 - r / rc) ** k * np.exp(-(r - c) ** 2 / (2 * w * w)), a, b)
                   for k in range(kmax + 1)])
    scale = np.abs(jq).max() + 1e-300
    assert np.all(np.abs(jr - jq) <= 1e-12 * scale + 1e-10 * np.abs(jq))


HP = [
    dict(sigma_r0=0.5, sigma_p0=0.5, alpha_r=0.0, alpha_p=0.0, amp_a=1.0),
    dict(sigma_r0=0.2, sigma_p0=0.4, alpha_r=0.08, alpha_p=0.08, amp_a=1.0),
    dict(sigma_r0=0.12, sigma_p0=0.55, alpha_r=0.14, alpha_p=0.06, amp_a=1.6),
    dict(sigma_r0=0.5, sigma_p0=0.5, alpha_r=0.0, alpha_p=0.0, amp_a=0.0),
]


@pytest.mark.parametrize("hp", HP)
@pytest.mark.parametrize("buffer", [0.0, 0.5, 1.2])
def test_radial_coefficients_eq01_by_quadrature(hp, buffer):
    # Eq. 01 in the primitive basis: A_j int_0^rc phi_a f(r) exp(-(r-r_j)^2/2 sr^2) dr;
    # the Gaussian row is the [0, inf) closed form without f (Sec. III.A)
    rc, n_max = 4.5, 7
    P = Params(r_cut=rc, r_soft=rc - buffer, n_max=n_max, l_max=2, **hp)
    rj = np.array([0.0, 0.4, 1.3, 2.9, 3.7, 4.1, 4.45])
    b = soap.radial_coefficients(torch.as_tensor(rj, dtype=DT), P).numpy()
    for t, x in enumerate(rj):
        sr = hp["sigma_r0"] + hp["alpha_r"] * x
        sp = hp["sigma_p0"] + hp["alpha_p"] * x
        u = x / rc
        amp = (1 + 2 * u ** 3 - 3 * u ** 2) ** hp["amp_a"] / (sr * sp * sp)
        fr = lambda r: soap.smoothing_function(torch.as_tensor(r), P).numpy()
        for a in range(1, n_max):
            integrand = (lambda r: basis.basis_functions(r, n_max, rc, hp["sigma_r0"])[a - 1]
                         * fr(r) * np.exp(-(r - x) ** 2 / (2 * sr * sr)))
            # split at r_soft, where f has a jump in its second derivative
            ref = amp * (quad(integrand, 0.0, P.r_soft) + (quad(integrand, P.r_soft, rc)
                                                           if buffer > 0 else 0.0))
            assert abs(b[t, a - 1] - ref) <= 1e-11 * max(abs(ref), 1e-3 * amp)
        ref = amp * quad(lambda r: basis.basis_functions(r, n_max, rc, hp["sigma_r0"])[-1]
                         * np.exp(-(r - x) ** 2 / (2 * sr * sr)), 0.0, 40.0, panels=800)
        assert abs(b[t, -1] - ref) <= 1e-11 * max(abs(ref), 1e-3 * amp)


def test_amplitude_and_its_slope_vanish_at_cutoff():
    # Eq. 15: the cubic goes from 1 at the origin to 0 at r_cut; for a >= 1 its slope too
    P = Params(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, amp_a=1.0)
    r = torch.tensor([0.0, 5.0 - 1e-4, 5.0 - 2e-4], dtype=DT)
    _, _, a = soap.widths_and_amplitude(r, P)
    assert float(a[0]) == pytest.approx(1.0 / 0.125)
    slope = (a[1] - a[2]) / 1e-4
    assert abs(float(a[1])) < 1e-6 and abs(float(slope)) < 1e-2
