"""Pins of the oracle's expansion coefficients, power spectrum and descriptor.

* c_nlm against brute-force quadrature of the model density (Eqs. 05, 15 and the
  smoothing of Sec. III.B) projected on g_n(r) Y_lm(r_hat) with measure dr dOmega;
* Eq. 09 against the full sum over m = -l..l built from a library Y_lm;
* the single-neighbour closed form of p, rotation/reflection/permutation invariance,
  smooth decay at r_cut, and the rotation-averaged overlap identity behind Eq. 03.
"""
import math

import numpy as np
import pytest
import scipy.special as sps
import torch

import synth
from oracle import Params, basis, soap

DT = torch.float64


def cluster(nbrs, side=40.0, species=None):
    """One centre at the middle of a large box plus neighbours at the given offsets."""
    c = np.full(3, side / 2)
    pos = np.vstack([c, c + np.asarray(nbrs, dtype=np.float64)])
    sp = np.zeros(len(pos), np.int32) if species is None else np.asarray(species, np.int32)
    return synth.concat([synth.Structure(pos=pos, cell=np.eye(3) * side, species=sp)])


P_QUAD = Params(r_cut=4.0, r_soft=3.4, sigma_r0=0.5, sigma_p0=0.6, alpha_r=0.05,
                alpha_p=0.03, amp_a=1.0, n_f=4.0, central_weight=0.0, n_max=5, l_max=5)

NEIGHBOUR_SETS = [
    [[1.1, 0.4, -0.7]],
    [[1.1, 0.4, -0.7], [-0.3, 2.2, 1.9]],
    [[1.1, 0.4, -0.7], [-0.3, 2.2, 1.9], [0.2, -3.1, 1.75]],
]


def sphere_grid(nt=64, nphi=128):
    ct, wt = np.polynomial.legendre.leggauss(nt)
    phis = 2 * np.pi * np.arange(nphi) / nphi
    theta = np.repeat(np.arccos(ct), nphi)
    phi = np.tile(phis, nt)
    w = np.repeat(wt, nphi) * (2 * np.pi / nphi)
    u = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], 1)
    return theta, phi, u, w


@pytest.mark.parametrize("k", range(len(NEIGHBOUR_SETS)))
@pytest.mark.parametrize("central", [0.0, 1.0])
def test_coefficients_by_3d_quadrature(k, central):
    P = Params(**{**P_QUAD.__dict__, "central_weight": central})
    nbrs = np.array(NEIGHBOUR_SETS[k])
    d = soap.descriptors(cluster(nbrs), P, centers=[0])
    c = (d["c_re"] - 1j * 0 + 1j * d["c_im"]).numpy()[0]        # [n, l, m]
    W = d["W"]
    rq, wr = basis.gauss_legendre(0.0, P.r_cut, panels=200, order=16)
    g = W @ basis.basis_functions(rq, P.n_max, P.r_cut, P.sigma_r0)   # [n, Nr]
    f = soap.smoothing_function(torch.as_tensor(rq), P).numpy()
    theta, phi, u, wa = sphere_grid()
    ylm_conj = {(l, m): np.conj(sps.sph_harm_y(l, m, theta, phi))
                for l in range(P.l_max + 1) for m in range(l + 1)}
    ref = np.zeros_like(c)
    sources = [(np.linalg.norm(v), v / np.linalg.norm(v)) for v in nbrs]
    for rj, uj in sources:
        sr = P.sigma_r0 + P.alpha_r * rj
        sp = P.sigma_p0 + P.alpha_p * rj
        x = rj / P.r_cut
        amp = (1 + 2 * x ** 3 - 3 * x ** 2) ** P.amp_a / (sr * sp * sp)
        radial = amp * f * np.exp(-(rq - rj) ** 2 / (2 * sr * sr))        # Eq. 05 (1)
        z = rj * rj / (sp * sp)
        angular = np.exp(-z) * np.exp(z * (u @ uj))                       # Eq. 05 (2)(3)
        bn = g @ (wr * radial)
        for (l, m), y in ylm_conj.items():
            ref[:, l, m] += bn * np.sum(wa * angular * y)
    if central:
        radial0 = (1.0 / (P.sigma_r0 * P.sigma_p0 ** 2)) * f * np.exp(-rq ** 2 / (2 * P.sigma_r0 ** 2))
        ref[:, 0, 0] += central * (g @ (wr * radial0)) * np.sum(wa * ylm_conj[(0, 0)])
    scale = np.abs(ref).max()
    assert np.abs(c - ref).max() < 1e-10 * scale


def test_eq08_weight_option_scales_by_2l_plus_1():
    nbrs = NEIGHBOUR_SETS[2]
    a = soap.descriptors(cluster(nbrs), P_QUAD, centers=[0])
    b = soap.descriptors(cluster(nbrs), Params(**{**P_QUAD.__dict__, "eq08_weight": True}),
                         centers=[0])
    w = torch.as_tensor([2 * l + 1 for l in range(P_QUAD.l_max + 1)], dtype=DT)
    assert torch.allclose(b["c_re"], a["c_re"] * w[None, None, :, None], rtol=1e-14, atol=1e-300)


def test_eq09_matches_full_m_sum():
    P = Params(**{**P_QUAD.__dict__, "central_weight": 1.0})
    nbrs = np.array(NEIGHBOUR_SETS[2])
    d = soap.descriptors(cluster(nbrs), P, centers=[0])
    W = d["W"]
    rj = torch.as_tensor(np.linalg.norm(nbrs, axis=1), dtype=DT)
    bn = (soap.radial_coefficients(rj, P) @ torch.as_tensor(W).T).numpy()
    _, sp, _ = soap.widths_and_amplitude(rj, P)
    il = soap.ilexp(rj * rj / (sp * sp), P.l_max).numpy()
    u = nbrs / np.linalg.norm(nbrs, axis=1, keepdims=True)
    th, ph = np.arccos(u[:, 2]), np.arctan2(u[:, 1], u[:, 0])
    b0 = (soap.radial_coefficients(torch.zeros(1, dtype=DT), P) @ torch.as_tensor(W).T).numpy()[0]
    p_full = np.zeros((P.n_max, P.n_max, P.l_max + 1))
    for l in range(P.l_max + 1):
        for m in range(-l, l + 1):
            cm = np.zeros(P.n_max, dtype=complex)
            for t in range(len(nbrs)):
                cm += 4 * np.pi * bn[t] * il[t, l] * np.conj(sps.sph_harm_y(l, m, th[t], ph[t]))
            if l == 0:
                cm += math.sqrt(4 * math.pi) * b0
            p_full[:, :, l] += np.real(np.outer(cm, np.conj(cm)))
    assert np.allclose(d["p"].numpy()[0], p_full, rtol=1e-12, atol=1e-12 * np.abs(p_full).max())


def test_single_neighbour_closed_form():
    # one neighbour, no central atom: p_nn'l = 4 pi (2l+1) b_n b_n' ilexp_l^2
    v = np.array([0.9, -1.3, 1.6])
    d = soap.descriptors(cluster([v]), P_QUAD, centers=[0])
    rj = torch.tensor([np.linalg.norm(v)], dtype=DT)
    bn = (soap.radial_coefficients(rj, P_QUAD) @ torch.as_tensor(d["W"]).T).numpy()[0]
    _, sp, _ = soap.widths_and_amplitude(rj, P_QUAD)
    il = soap.ilexp(rj * rj / (sp * sp), P_QUAD.l_max).numpy()[0]
    ref = np.einsum("a,b,l->abl", bn, bn, 4 * np.pi * (2 * np.arange(P_QUAD.l_max + 1) + 1) * il ** 2)
    assert np.allclose(d["p"].numpy()[0], ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def box_params():
    return Params(r_cut=3.7, r_soft=3.2, sigma_r0=0.5, sigma_p0=0.5, n_max=6, l_max=6,
                  n_species=2)


@pytest.mark.parametrize("reflect", [False, True])
def test_rotation_and_reflection_invariance(reflect):
    s = synth.random_box(24, side=6.0, dmin=1.2, seed=11, species_probs=(0.6, 0.4), shear=0.15)
    R = synth.random_rotation(5, reflect=reflect)
    a = soap.descriptors(synth.concat([s]), box_params())
    s2 = synth.Structure(pos=s.pos @ R.T, cell=s.cell @ R.T, species=s.species)
    b = soap.descriptors(synth.concat([s2]), box_params())
    assert np.array_equal(a["pairs"]["j"], b["pairs"]["j"])
    rel = (a["p"] - b["p"]).flatten(1).norm(dim=1) / a["p"].flatten(1).norm(dim=1)
    assert float(rel.max()) < 1e-12


def test_permutation_invariance():
    s = synth.random_box(24, side=6.0, dmin=1.2, seed=12, species_probs=(0.6, 0.4))
    perm = np.random.default_rng(0).permutation(24)
    a = soap.descriptors(synth.concat([s]), box_params())
    s2 = synth.Structure(pos=s.pos[perm], cell=s.cell, species=s.species[perm])
    b = soap.descriptors(synth.concat([s2]), box_params())
    rel = (a["p"][perm] - b["p"]).flatten(1).norm(dim=1) / b["p"].flatten(1).norm(dim=1)
    assert float(rel.max()) < 1e-12


def test_contribution_and_slope_vanish_at_cutoff():
    # with a = 1 (Eq. 15) a neighbour's coefficients fall like (r_cut - r)^2 near r_cut
    u = np.array([0.3, -0.5, 0.81])
    u = u / np.linalg.norm(u)
    norms = []
    for delta in (1e-2, 1e-3):
        d = soap.descriptors(cluster([u * (P_QUAD.r_cut - delta)]), P_QUAD, centers=[0])
        norms.append(float(torch.sqrt((d["c_re"] ** 2 + d["c_im"] ** 2).sum())))
    assert norms[1] / norms[0] == pytest.approx(1e-2, rel=0.05)


def euler(a, b, g):
    def rz(t):
        c, s = math.cos(t), math.sin(t)
        return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])

    def ry(t):
        c, s = math.cos(t), math.sin(t)
        return np.array([[c, 0, s], [0, 1.0, 0], [-s, 0, c]])
    return rz(a) @ ry(b) @ rz(g)


def test_rotation_averaged_overlap_identity():
    # Sec. I, Eq. 03: int dR |<rho_i | R rho_j>|^2 = sum_l 8 pi^2/(2l+1) sum_nn' p_nn'l(i) p_nn'l(j)
    P = Params(r_cut=4.0, r_soft=3.5, sigma_r0=0.5, sigma_p0=0.5, n_max=3, l_max=3,
               central_weight=1.0)
    env_i = np.array([[1.2, 0.3, -0.4], [-0.6, 1.9, 0.8], [0.1, -0.7, -2.4]])
    env_j = np.array([[-1.0, 1.1, 0.2], [2.1, 0.4, 1.3], [0.5, -2.2, 0.9], [-0.8, -0.5, -1.6]])
    lm = P.l_max
    na, ng = 4 * lm + 2, 4 * lm + 2
    xb, wb = np.polynomial.legendre.leggauss(2 * lm + 2)
    rots, wts = [], []
    for ia in range(na):
        for ib, cb in enumerate(xb):
            for ig in range(ng):
                rots.append(euler(2 * np.pi * ia / na, math.acos(cb), 2 * np.pi * ig / ng))
                wts.append((2 * np.pi / na) * wb[ib] * (2 * np.pi / ng))
    structs = [cluster(env_i).structure(0)] + [cluster(env_j @ R.T).structure(0) for R in rots]
    batch = synth.concat(structs)
    centers = batch.atom_offs[:-1]
    d = soap.descriptors(batch, P, centers=centers)
    cre, cim = d["c_re"].numpy(), d["c_im"].numpy()
    wm = np.array([1.0] + [2.0] * lm)
    ov = np.einsum("nlm,rnlm,m->r", cre[0], cre[1:], wm) + np.einsum("nlm,rnlm,m->r", cim[0], cim[1:], wm)
    lhs = np.sum(np.array(wts) * ov ** 2)
    dj = soap.descriptors(cluster(env_j), P, centers=[0])
    pi_, pj = d["p"].numpy()[0], dj["p"].numpy()[0]
    rhs = sum(8 * np.pi ** 2 / (2 * l + 1) * np.sum(pi_[:, :, l] * pj[:, :, l]) for l in range(lm + 1))
    assert lhs == pytest.approx(rhs, rel=1e-11)


def test_packed_layout_preserves_dot_products():
    s = synth.random_box(24, side=6.0, dmin=1.2, seed=13, species_probs=(0.6, 0.4))
    d = soap.descriptors(synth.concat([s]), box_params())
    p = d["p"]
    q = d["q"]
    full = torch.einsum("iabl,jabl->ij", p, p) / (d["pnorm"][:, None] * d["pnorm"][None, :])
    assert torch.allclose(q @ q.T, full, rtol=1e-13, atol=1e-15)
    assert torch.allclose(soap.unpack(soap.pack(p), p.shape[1], p.shape[3] - 1), p, rtol=1e-14)
    assert q.shape[1] == box_params().dim
