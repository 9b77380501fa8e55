"""The column layout of the fitting-matrix force rows, on the oracle's pair lists (no GPU).

Columns are stored by target atom: the pair (j -> k, S) fills the slot of its reverse
(k -> j, -S) in k's range, and k's three self columns follow its pairs, so atom k owns
columns [3 (o_k + k), 3 (o_(k+1) + k + 1)) with o_k its first pair in the list.  The layout
must be a bijection onto [0, 3 (P + N)) whose column ranges are contiguous per target; and
summing, per target, the contributions placed there must give the derivative of the
per-structure kernel sums (checked against the oracle's kernel_gradients).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import Params, basis, gap, neighbours, soap


def pair_list(batch, r_cut):
    pr = neighbours.batch_pairs(batch, r_cut)
    i, j, S = pr["i"], pr["j"], pr["shift"]
    key = {(int(a), int(b), tuple(int(x) for x in s)): p for p, (a, b, s) in enumerate(zip(i, j, S))}
    rev = np.array([key[(int(b), int(a), tuple(-int(x) for x in s))] for a, b, s in zip(i, j, S)])
    offs = np.searchsorted(i, np.arange(batch.n_atoms + 1))
    return pr, rev, offs


def columns(pr, rev, offs, n):
    """(column of each pair's first component, column of each atom's first self component)."""
    pair_col = 3 * (rev + pr["j"])
    self_col = 3 * (offs[1:] + np.arange(n))
    return pair_col, self_col


@pytest.mark.parametrize("case", ["box", "self_images", "ragged"])
def test_layout_is_a_bijection_with_contiguous_targets(case):
    if case == "box":
        batch, r_cut = synth.get_workload("box64_n6l6").structures(), 3.7
    elif case == "self_images":
        batch, r_cut = synth.concat([synth.random_box(7, side=3.1, dmin=1.0, seed=5, shear=0.35)]), 5.0
    else:
        batch, r_cut = synth.batched_boxes(6, n_lo=1, n_hi=40, seed=12), 4.5
    pr, rev, offs = pair_list(batch, r_cut)
    n, P = batch.n_atoms, len(pr["i"])
    pair_col, self_col = columns(pr, rev, offs, n)
    cols = np.concatenate([pair_col[:, None] + np.arange(3), self_col[:, None] + np.arange(3)]).ravel()
    assert np.array_equal(np.sort(cols), np.arange(3 * (P + n)))
    # each target's columns form one range: its pairs' slots, then its self slot
    target = np.concatenate([np.repeat(pr["j"], 3), np.repeat(np.arange(n), 3)])
    order = np.argsort(cols)
    assert np.all(np.diff(target[order]) >= 0)
    for k in range(n):
        lo, hi = 3 * (offs[k] + k), 3 * (offs[k + 1] + k + 1)
        assert np.all(target[order][lo:hi] == k)


def test_target_sums_give_the_force_rows():
    """Scatter the per-pair contributions w_is (q_s - S_is q_i) . dp_i/dr_ij into the layout,
    sum each target's range, and compare with the oracle's kernel_gradients."""
    batch = synth.concat([synth.random_box(10, side=4.8, dmin=1.2, seed=8)])
    w = synth.get_workload("box64_n6l6")
    P = Params.from_dict(w.params())
    W = basis.orthonormaliser(P.n_max, P.r_cut, P.sigma_r0)
    sb = w.sparse_box()
    qs = torch.as_tensor(gap.sparse_set(sb, P, synth.sparse_indices(sb.n_atoms, 5, w.sparse_seed), W=W))
    zeta = 3.0
    pr, rev, offs = pair_list(batch, P.r_cut)
    n, npair = batch.n_atoms, len(pr["i"])
    # dp_i/dr_ij per pair by autograd on the pair vectors
    pos = torch.as_tensor(batch.pos)
    cell = torch.as_tensor(batch.cell)
    rvec = soap.pair_vectors(pos, cell, pr).detach().clone().requires_grad_(True)
    orig = soap.pair_vectors
    try:
        soap.pair_vectors = lambda *_: rvec
        c_re, c_im = soap.expansion_coefficients(P, W, pos, cell, batch.species, np.arange(n), pr)
    finally:
        soap.pair_vectors = orig
    p = soap.pack(soap.power_spectrum(c_re, c_im))            # [n, D]
    pn = p.norm(dim=1)
    q = (p / pn[:, None]).detach()
    S = q @ qs.T                                               # [n, M]
    wts = zeta * S ** (zeta - 1) / pn.detach()[:, None]
    contrib = torch.zeros(npair, 3, len(qs), dtype=torch.float64)   # dk(i, s)/dr_ij
    for s in range(len(qs)):
        u = wts[:, s:s + 1] * (qs[s][None, :] - S[:, s:s + 1] * q)    # [n, D]
        g, = torch.autograd.grad((p * u).sum(), rvec, retain_graph=True)
        contrib[:, :, s] = g
    pair_col, self_col = columns(pr, rev, offs, n)
    ncols = 3 * (npair + n)
    colv = torch.zeros(ncols, len(qs), dtype=torch.float64)
    target = np.zeros(ncols, dtype=np.int64)
    for p_ in range(npair):
        colv[pair_col[p_]:pair_col[p_] + 3] = contrib[p_]
        target[pair_col[p_]:pair_col[p_] + 3] = pr["j"][p_]
    for k in range(n):
        own = torch.as_tensor(pr["i"] == k)
        colv[self_col[k]:self_col[k] + 3] = -contrib[own].sum(dim=0)
        target[self_col[k]:self_col[k] + 3] = k
    dk = np.zeros((n, 3, len(qs)))
    for k in range(n):
        lo, hi = 3 * (offs[k] + k), 3 * (offs[k + 1] + k + 1)
        assert np.all(target[lo:hi] == k)
        dk[k] = colv[lo:hi].reshape(-1, 3, len(qs)).sum(dim=0).numpy()
    ref = gap.kernel_gradients(batch, P, qs.numpy(), zeta, W=W)
    assert np.allclose(dk, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
