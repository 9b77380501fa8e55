"""Pins of the oracle's angular functions: ilexp (Sec. III.C) and Y_lm (Sec. III.C)."""
import math

import numpy as np
import pytest
import scipy.special as sps
import torch

from oracle import basis, soap

DT = torch.float64
ZS = [1e-6, 1e-3, 0.3, 2.0, 5.76, 10.0, 25.0, 39.99, 40.01, 64.0, 100.0, 289.0, 1700.0]


def test_ilexp_closed_forms_l0_l1(golden):
    # the paper's closed forms for l = 0, 1 (checked at z = x^2 away from 0)
    g = golden["ilexp_closed_forms"]
    z = torch.tensor([z for z in ZS if z > 0.1], dtype=DT)
    il = soap.ilexp(z, 1).numpy()
    for k, zz in enumerate(z.numpy()):
        x = math.sqrt(zz)
        l0 = eval(g["l0"].replace("^", "**"), {"x": x, "exp": math.exp})
        l1 = eval(g["l1"].replace("^", "**"), {"x": x, "exp": math.exp})
        assert il[k, 0] == pytest.approx(l0, rel=1e-14)
        assert il[k, 1] == pytest.approx(l1, rel=1e-12)


def test_ilexp_small_x_limits():
    # Sec. III.C: ilexp(x;0) -> 1 - x^2 and ilexp(x;l) -> x^(2l)/(2l+1)!! as x -> 0
    x = 1e-3
    il = soap.ilexp(torch.tensor([x * x], dtype=DT), 12).numpy()[0]
    assert abs(il[0] - (1 - x * x)) < 1e-11
    for l in range(1, 13):
        df = np.prod(np.arange(2 * l + 1, 0, -2, dtype=np.float64))
        assert il[l] == pytest.approx(x ** (2 * l) / df, rel=1e-5)


def test_ilexp_integral_representation():
    # e^{-z} i_l(z) = 1/2 int_{-1}^{1} e^{z(t-1)} P_l(t) dt (from the Kaufmann expansion
    # e^{z cos e} = sum (2l+1) i_l(z) P_l(cos e) and orthogonality of P_l)
    t, w = basis.gauss_legendre(-1.0, 1.0, panels=400, order=20)
    z = np.array([0.3, 2.0, 10.0, 39.0, 41.0, 100.0])
    il = soap.ilexp(torch.as_tensor(z, dtype=DT), 12).numpy()
    for l in range(13):
        pl = np.polynomial.legendre.legval(t, [0] * l + [1])
        ref = np.array([0.5 * np.sum(w * np.exp(zz * (t - 1)) * pl) for zz in z])
        # the quadrature of an oscillating integrand carries an absolute error near 1e-16
        assert np.allclose(il[:, l], ref, rtol=1e-9, atol=1e-14)


def test_ilexp_against_library_bessel():
    z = np.array([zz for zz in ZS if zz < 600])
    il = soap.ilexp(torch.as_tensor(z, dtype=DT), 12).numpy()
    for l in range(13):
        ref = sps.spherical_in(l, z) * np.exp(-z)
        assert np.allclose(il[:, l], ref, rtol=1e-13, atol=0)


def test_ilexp_paper_recursion_where_well_conditioned():
    # Sec. III.C upward recursion ilexp(l) = ilexp(l-2) - (2l-1)/x^2 ilexp(l-1), started
    # from the closed forms; it is well conditioned for x^2 >> l^2
    z = torch.tensor([300.0, 1000.0, 1700.0], dtype=DT)
    il = soap.ilexp(z, 12).numpy()
    rec = [il[:, 0], il[:, 1]]
    for l in range(2, 13):
        rec.append(rec[l - 2] - (2 * l - 1) / z.numpy() * rec[l - 1])
    assert np.allclose(np.stack(rec, 1), il, rtol=1e-12)


def test_ilexp_continuous_across_branch():
    z = torch.tensor([soap.ILEXP_SERIES_MAX_Z * (1 - 1e-12), soap.ILEXP_SERIES_MAX_Z * (1 + 1e-12)],
                     dtype=DT)
    il = soap.ilexp(z, 12).numpy()
    assert np.allclose(il[0], il[1], rtol=1e-13)


def test_legendre_seeds(golden):
    # the six tabulated starting polynomials of Sec. III.C
    xs = np.array([-0.93, -0.2, 0.0, 0.41, 0.77])
    p = soap.associated_legendre(torch.as_tensor(xs, dtype=DT), 2).numpy()
    env = {"sqrt": np.sqrt}
    for name, expr in golden["legendre_seeds"]["polynomials"].items():
        l, m = int(name[1]), int(name[2])
        ref = eval(expr.replace("^", "**"), dict(env, x=xs))
        assert np.allclose(p[:, l, m], ref * np.ones_like(xs), atol=1e-15)


def random_dirs(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_conj_harmonics_match_library():
    u = random_dirs(50, 1)
    re, im = soap.conj_spherical_harmonics(torch.as_tensor(u, dtype=DT), 12)
    theta = np.arccos(u[:, 2])
    phi = np.arctan2(u[:, 1], u[:, 0])
    for l in range(13):
        for m in range(l + 1):
            ref = np.conj(sps.sph_harm_y(l, m, theta, phi))
            assert np.allclose(re[:, l, m].numpy(), ref.real, atol=1e-13)
            assert np.allclose(im[:, l, m].numpy(), ref.imag, atol=1e-13)


def test_addition_theorem():
    # sum_m Y_lm(a) Y*_lm(b) = (2l+1)/(4 pi) P_l(a.b); with m >= 0 values only:
    # Y_l0(a)Y_l0(b) + 2 sum_{m>=1} Re(Y_lm(a) Y*_lm(b))
    a, b = random_dirs(20, 2), random_dirs(20, 3)
    ra, ia = soap.conj_spherical_harmonics(torch.as_tensor(a, dtype=DT), 10)
    rb, ib = soap.conj_spherical_harmonics(torch.as_tensor(b, dtype=DT), 10)
    cosg = np.sum(a * b, axis=1)
    for l in range(11):
        w = np.array([1.0] + [2.0] * l)
        lhs = np.sum(w[None] * (ra[:, l, :l + 1] * rb[:, l, :l + 1]
                                + ia[:, l, :l + 1] * ib[:, l, :l + 1]).numpy(), axis=1)
        rhs = (2 * l + 1) / (4 * np.pi) * np.polynomial.legendre.legval(cosg, [0] * l + [1])
        assert np.allclose(lhs, rhs, atol=1e-13)


def test_orthonormality_on_sphere():
    ct, wt = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phis = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - ct * ct)
    u = np.stack([np.outer(st, np.cos(phis)), np.outer(st, np.sin(phis)),
                  np.outer(ct, np.ones(nphi))], -1).reshape(-1, 3)
    w = np.outer(wt, np.full(nphi, 2 * np.pi / nphi)).reshape(-1)
    re, im = soap.conj_spherical_harmonics(torch.as_tensor(u, dtype=DT), 8)
    y = (re - 1j * im).numpy().reshape(len(u), -1)     # Y_lm, m >= 0, flattened (l, m)
    gram = (y.conj().T * w[None]) @ y
    idx = [(l, m) for l in range(9) for m in range(9)]
    for a, (l, m) in enumerate(idx):
        for b, (l2, m2) in enumerate(idx):
            if m > l or m2 > l2:
                continue
            ref = 1.0 if (l, m) == (l2, m2) else 0.0
            assert abs(gram[a, b] - ref) < 1e-12
