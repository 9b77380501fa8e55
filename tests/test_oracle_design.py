"""Pins of the oracle's sparse-GAP fitting matrices (Sec. IV.A with the kernel of Sec. I).

  kernel_matrix     K_MM of a sparse set has a unit diagonal, is symmetric and positive
                    semi-definite (for integer zeta it is a Hadamard power of a Gram
                    matrix); K_NM alpha equals the local energies of the model evaluation
  structure_rows    rows summed per structure equal the model's structure energies
  kernel_gradients  central finite differences of the per-structure kernel sums; the force
                    identity F = -dk alpha against the model evaluation (itself pinned by
                    finite differences); zero sum over each structure (translation
                    invariance); rotation covariance; restricted evaluation (sampled atoms
                    and sparse columns) equal to the full one
"""
import numpy as np
import pytest
import torch

import synth
from oracle import Params, gap, soap

DT = torch.float64


@pytest.fixture(scope="module")
def setup():
    w = synth.get_workload("box64_n6l6")
    P = Params.from_dict(w.params())
    sb = w.sparse_box()
    m = 12
    qs = gap.sparse_set(sb, P, synth.sparse_indices(sb.n_atoms, m, w.sparse_seed))
    al = synth.gap_weights(m, w.alpha_seed)
    # two small structures of different shapes: per-structure sums must not mix them
    batch = synth.concat([synth.random_box(14, side=5.0, dmin=1.2, seed=31, shear=0.1),
                          synth.random_box(9, side=4.6, dmin=1.2, seed=32)])
    dk = gap.kernel_gradients(batch, P, qs, 4.0)
    return P, qs, al, batch, dk


def test_sparse_covariance_is_a_kernel_matrix(setup):
    P, qs, al, batch, dk = setup
    for zeta in (1.0, 2.0, 4.0):
        k = gap.kernel_matrix(qs, qs, zeta)
        assert torch.allclose(torch.diagonal(k), torch.ones(len(qs), dtype=DT), atol=1e-14)
        assert torch.allclose(k, k.T, atol=0, rtol=0)
        assert float(torch.linalg.eigvalsh(k).min()) > -1e-12 * len(qs)
        assert float(k.min()) >= 0.0 and float(k.max()) <= 1.0 + 1e-14


def test_kernel_rows_reproduce_model_energies(setup):
    P, qs, al, batch, dk = setup
    q = soap.descriptors(batch, P)["q"]
    k = gap.kernel_matrix(q, qs, 4.0)
    r = gap.evaluate(batch, P, qs, al, 4.0, forces=False, virial=False)
    assert np.allclose((k @ torch.as_tensor(al)).numpy(), r["e_atom"], rtol=1e-13, atol=1e-15)
    ks = gap.structure_rows(k, batch.atom_offs)
    assert ks.shape == (batch.n_struct, len(qs))
    assert np.allclose((ks @ torch.as_tensor(al)).numpy(), r["e_struct"], rtol=1e-13)


def struct_kernel_sum(batch, P, qs, zeta, t):
    q = soap.descriptors(batch, P)["q"]
    k = gap.kernel_matrix(q, qs, zeta)
    return gap.structure_rows(k, batch.atom_offs)[t].numpy()


def test_kernel_gradients_by_central_differences(setup):
    P, qs, al, batch, dk = setup
    h = 1e-5
    struct_of = np.repeat(np.arange(batch.n_struct), np.diff(batch.atom_offs))
    for atom, comp in [(0, 0), (5, 2), (13, 1), (14, 0), (20, 2)]:
        vals = []
        for sgn in (1, -1):
            pos = batch.pos.copy()
            pos[atom, comp] += sgn * h
            b = synth.Batch(pos, batch.cell, batch.species, batch.atom_offs)
            vals.append(struct_kernel_sum(b, P, qs, 4.0, struct_of[atom]))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert np.allclose(dk[atom, comp], fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())


def test_force_identity(setup):
    P, qs, al, batch, dk = setup
    r = gap.evaluate(batch, P, qs, al, 4.0, virial=False)
    f = -(dk @ al)
    assert np.allclose(f, r["forces"], rtol=1e-10, atol=1e-12 * np.abs(r["forces"]).max())


def test_translation_invariance_per_structure(setup):
    P, qs, al, batch, dk = setup
    scale = np.abs(dk).max()
    for t in range(batch.n_struct):
        a, b = batch.atom_offs[t], batch.atom_offs[t + 1]
        assert np.abs(dk[a:b].sum(axis=0)).max() < 1e-11 * scale


def test_rotation_covariance(setup):
    P, qs, al, batch, dk = setup
    rot = synth.random_rotation(7)
    b = synth.Batch(batch.pos @ rot.T, batch.cell @ rot.T, batch.species, batch.atom_offs)
    dk_rot = gap.kernel_gradients(b, P, qs, 4.0)
    assert np.allclose(dk_rot, np.einsum("ab,kbs->kas", rot, dk), rtol=1e-9,
                       atol=1e-11 * np.abs(dk).max())


def test_restricted_evaluation_matches_full(setup):
    P, qs, al, batch, dk = setup
    atoms, sparse = np.array([3, 16, 4]), np.array([7, 0])
    part = gap.kernel_gradients(batch, P, qs, 4.0, atoms=atoms, sparse=sparse)
    assert np.allclose(part, dk[atoms][:, :, sparse], rtol=1e-12, atol=1e-14 * np.abs(dk).max())
