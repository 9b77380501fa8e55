"""Pins of the oracle's GAP energy, forces, virial (Sec. IV.A) and neighbour search.

Forces and virial are checked against central finite differences of the energy
(h = 1e-5 A and a 2e-5 strain), translation invariance and symmetry; the kernel
against its bounds; the neighbour search against a naive triple loop over images.
"""
import itertools

import numpy as np
import pytest
import torch

import synth
from oracle import Params, gap, neighbours, soap

DT = torch.float64


@pytest.fixture(scope="module")
def model():
    w = synth.get_workload("box64_n6l6")
    P = Params.from_dict(w.params())
    sb = w.sparse_box()
    qs = gap.sparse_set(sb, P, synth.sparse_indices(sb.n_atoms, 16, w.sparse_seed))
    al = synth.gap_weights(16, w.alpha_seed)
    box = synth.random_box(20, side=5.5, dmin=1.2, seed=21, shear=0.1)
    return P, qs, al, synth.concat([box])


def energy(batch, P, qs, al, zeta):
    return gap.evaluate(batch, P, qs, al, zeta, forces=False, virial=False)["e_struct"].sum()


def test_kernel_bounds_and_self_similarity(model):
    P, qs, al, b = model
    q = soap.descriptors(b, P)["q"]
    k = q @ q.T
    assert torch.allclose(torch.diagonal(k), torch.ones(len(q), dtype=DT), atol=1e-14)
    assert float(k.min()) >= 0.0 and float(k.max()) <= 1.0 + 1e-14


def test_zeta_one_is_linear(model):
    P, qs, al, b = model
    q = soap.descriptors(b, P)["q"]
    e = gap.local_energies(q, torch.as_tensor(qs), torch.as_tensor(al), 1.0)
    assert torch.allclose(e, q @ (torch.as_tensor(qs).T @ torch.as_tensor(al)), rtol=1e-13)


@pytest.mark.parametrize("s,zeta,expected", [
    (0.5, 4.0, 0.0625),                 # 2^-4
    (0.5, 2.0, 0.25),                   # 2^-2
    (0.5, 2.5, 2.0 ** -2.5),            # 0.17677669529663687
    (0.25, 0.5, 0.5),                   # square root
    (0.9, 3.0, 0.729),                  # 0.9 * 0.9 * 0.9
    (1.0, 7.0, 1.0),                    # a unit self-similarity stays 1
    (0.0, 4.0, 0.0),
    (-1e-17, 2.5, 0.0),                 # a rounding-negative dot product is clamped (non-integer zeta)
    (-0.5, 3.0, -0.125),                # integer zeta: plain repeated product, sign kept
])
def test_kernel_power_hand_values(s, zeta, expected):
    """(q_i . q_s)^zeta of the SOAP kernel (Sec. I) at values fixed by arithmetic alone:
    a wrong exponent (zeta - 1, zeta + 1) or a wrong branch fails at least one case."""
    got = float(gap.kernel_power(torch.tensor([s], dtype=DT), zeta)[0])
    assert got == pytest.approx(expected, rel=1e-15, abs=0.0)


def test_local_energies_by_hand():
    """eps_i = sum_s alpha_s (q_i . q_s)^zeta (Sec. IV.A) on two 2-dimensional unit
    descriptors and two sparse rows, summed by hand: q_0 . q_s = (1, 0.6), q_1 . q_s = (0, 0.8)."""
    q = torch.tensor([[1.0, 0.0], [0.0, 1.0]], dtype=DT)
    qs = torch.tensor([[1.0, 0.0], [0.6, 0.8]], dtype=DT)
    al = torch.tensor([0.5, -2.0], dtype=DT)
    e2 = gap.local_energies(q, qs, al, 2.0)
    assert e2.tolist() == pytest.approx([0.5 - 2.0 * 0.36, -2.0 * 0.64], rel=1e-15)
    e4 = gap.local_energies(q, qs, al, 4.0)
    assert e4.tolist() == pytest.approx([0.5 - 2.0 * 0.1296, -2.0 * 0.4096], rel=1e-15)
    e15 = gap.local_energies(q, qs, al, 1.5)
    assert e15.tolist() == pytest.approx([0.5 - 2.0 * 0.6 ** 1.5, -2.0 * 0.8 ** 1.5], rel=1e-15)


@pytest.mark.parametrize("zeta", [4.0, 2.5])
def test_forces_by_central_differences(model, zeta):
    P, qs, al, b = model
    r = gap.evaluate(b, P, qs, al, zeta)
    h = 1e-5
    for atom, comp in [(0, 0), (3, 1), (7, 2), (11, 0)]:
        vals = []
        for sgn in (1, -1):
            pos = b.pos.copy()
            pos[atom, comp] += sgn * h
            vals.append(energy(synth.Batch(pos, b.cell, b.species, b.atom_offs), P, qs, al, zeta))
        fd = -(vals[0] - vals[1]) / (2 * h)
        assert r["forces"][atom, comp] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_virial_by_central_differences(model):
    P, qs, al, b = model
    r = gap.evaluate(b, P, qs, al, 4.0)
    h = 2e-5
    for a, c in [(0, 0), (1, 2), (2, 1)]:
        vals = []
        for sgn in (1, -1):
            e = np.zeros((3, 3))
            e[a, c] = sgn * h
            m = np.eye(3) + e
            vals.append(energy(synth.Batch(b.pos @ m.T, b.cell @ m.T, b.species, b.atom_offs),
                               P, qs, al, 4.0))
        fd = -(vals[0] - vals[1]) / (2 * h)
        assert r["virial"][0, a, c] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_translation_invariance_and_symmetric_virial(model):
    P, qs, al, b = model
    r = gap.evaluate(b, P, qs, al, 4.0)
    assert np.abs(r["forces"].sum(0)).max() < 1e-12
    v = r["virial"][0]
    assert np.abs(v - v.T).max() < 1e-12 * np.abs(v).max()


def test_sampled_forces_equal_full_forces(model):
    P, qs, al, b = model
    r = gap.evaluate(b, P, qs, al, 4.0)
    f, atoms = gap.forces_at(b, P, qs, al, 4.0, [2, 5, 17])
    assert np.allclose(f, r["forces"][atoms], rtol=1e-12, atol=1e-14)


def naive_pairs(pos, cell, rc, nimg=5):
    out = set()
    for i in range(len(pos)):
        for j in range(len(pos)):
            for s in itertools.product(range(-nimg, nimg + 1), repeat=3):
                if i == j and s == (0, 0, 0):
                    continue
                d = pos[j] + np.array(s) @ cell - pos[i]
                if d @ d < rc * rc:
                    out.add((i, j, s))
    return out


@pytest.mark.parametrize("shear,rc", [(0.0, 3.7), (0.3, 4.5), (0.5, 2.0)])
def test_neighbour_search_against_naive_loop(shear, rc):
    s = synth.random_box(5, side=3.0, dmin=1.0, seed=7, shear=shear)
    i, j, S, r = neighbours.structure_pairs(s.pos, s.cell, s.species, rc)
    got = {(a, b, tuple(x)) for a, b, x in zip(i, j, S)}
    assert got == naive_pairs(s.pos, s.cell, rc)
    assert len(got) == len(i)


def test_neighbour_list_symmetric_and_canonical():
    s = synth.random_box(30, side=6.5, dmin=1.1, seed=8, shear=0.2, species_probs=(0.5, 0.5))
    i, j, S, r = neighbours.structure_pairs(s.pos, s.cell, s.species, 4.2)
    key = {(a, b, tuple(x)): k for k, (a, b, x) in enumerate(zip(i, j, S))}
    for k, (a, b, x) in enumerate(zip(i, j, S)):
        back = key[(b, a, tuple(-x))]
        assert np.array_equal(r[back], -r[k])
    order = np.lexsort((S[:, 2], S[:, 1], S[:, 0], j, s.species[j], i))
    assert np.array_equal(order, np.arange(len(i)))
    d2 = (r[:, 0] * r[:, 0] + r[:, 1] * r[:, 1]) + r[:, 2] * r[:, 2]
    assert d2.max() < 4.2 ** 2 and d2.min() > 0


def test_forces_with_self_images_on_the_axes(model):
    # a cubic cell smaller than r_cut puts periodic self-images exactly on the z axis (the
    # pole of the spherical harmonics); forces must stay finite and match differences
    P, qs, al, _ = model
    s = synth.random_box(3, side=3.2, dmin=1.0, seed=9)
    b = synth.concat([s])
    r = gap.evaluate(b, P, qs, al, 2.0)
    assert np.all(np.isfinite(r["forces"])) and np.all(np.isfinite(r["virial"]))
    h = 1e-5
    for atom, comp in [(0, 2), (1, 0)]:
        vals = []
        for sgn in (1, -1):
            pos = b.pos.copy()
            pos[atom, comp] += sgn * h
            vals.append(energy(synth.Batch(pos, b.cell, b.species, b.atom_offs), P, qs, al, 2.0))
        assert r["forces"][atom, comp] == pytest.approx(-(vals[0] - vals[1]) / (2 * h), rel=1e-6, abs=1e-9)
