"""The synthetic workloads follow their stated recipes (no GPU).

They stand in for the paper's amorphous-carbon and hydrogen-adsorption data (Sec. IV),
which are not available: seeded periodic cubes at a-C-like number densities with a
minimum atom distance, a batch of uneven cubes, and a random GAP model.  These tests
check that the generators produce what the recipes state, so that the parity and
throughput figures are about the stated workloads.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import synth

BOXES = ["box64_n6l6", "box1000_n8l8", "twospecies4096_n8l8", "box100k_n10l10"]
# cube edges implied by the stated atom counts and densities (A)
EDGES = {"box64_n6l6": 8.0, "box1000_n8l8": 18.82, "twospecies4096_n8l8": 34.47,
         "box100k_n10l10": 87.36}


def nearest_distances(pos, side):
    """Minimum-image distance of every atom to its nearest other atom in a cube."""
    p = np.mod(pos, side)
    d, _ = cKDTree(p, boxsize=side).query(p, k=2)
    return d[:, 1]


@pytest.fixture(scope="module")
def boxes():
    return {n: synth.get_workload(n).structures() for n in BOXES}


@pytest.mark.parametrize("name", BOXES)
def test_boxes_follow_their_recipe(boxes, name):
    w = synth.get_workload(name)
    b = boxes[name]
    assert b.n_struct == 1 and b.n_atoms == w.n_atoms
    side = b.cell[0, 0, 0]
    assert side == pytest.approx(EDGES[name], abs=5e-3)
    assert np.array_equal(b.cell[0], np.eye(3) * side)
    assert np.all(b.pos >= 0.0) and np.all(b.pos < side)
    assert nearest_distances(b.pos, side).min() >= w.dmin
    if w.species_probs is None:
        assert np.all(b.species == 0)
    else:
        p = np.asarray(w.species_probs)
        frac = np.bincount(b.species, minlength=len(p)) / b.n_atoms
        assert np.all(np.abs(frac - p) < 5 * np.sqrt(p * (1 - p) / b.n_atoms))


def test_batch_follows_its_recipe():
    w = synth.get_workload("batch256_n8l8")
    b = w.structures()
    assert b.n_struct == 256
    n = np.diff(b.atom_offs)
    assert n.min() >= w.n_lo and n.max() <= w.n_hi
    # log-uniform counts: ln N is uniform on [ln 16, ln 2000] (mean and spread within 4 sigma)
    lo, hi = np.log(w.n_lo), np.log(w.n_hi)
    ln = np.log(n)
    assert abs(ln.mean() - (lo + hi) / 2) < 4 * (hi - lo) / np.sqrt(12 * 256)
    assert ln.std() == pytest.approx((hi - lo) / np.sqrt(12), rel=0.15)
    edges = b.cell[:, 0, 0]
    rho = n / edges ** 3
    assert rho.min() >= w.rho_lo - 1e-12 and rho.max() <= w.rho_hi + 1e-12
    for s in range(0, 256, 16):                       # minimum distance on a sample of cubes
        pos = b.pos[b.atom_offs[s]:b.atom_offs[s + 1]]
        assert nearest_distances(pos, edges[s]).min() >= w.dmin


@pytest.mark.parametrize("name", ["box1000_n8l8", "twospecies4096_n8l8", "batch256_n8l8",
                                  "box100k_n10l10"])
def test_gap_model_inputs(name):
    w = synth.get_workload(name)
    sb = w.sparse_box()
    idx = synth.sparse_indices(sb.n_atoms, w.n_sparse, w.sparse_seed)
    assert len(np.unique(idx)) == w.n_sparse and idx.min() >= 0 and idx.max() < sb.n_atoms
    al = synth.gap_weights(w.n_sparse, w.alpha_seed)
    # alpha_s ~ N(0, 0.01): sample variance within 5 standard errors
    assert abs(al.var() - 0.01) < 5 * 0.01 * np.sqrt(2.0 / w.n_sparse)
    assert abs(al.mean()) < 5 * 0.1 / np.sqrt(w.n_sparse)


def test_generators_are_deterministic():
    a = synth.random_box(200, density=0.15, dmin=1.2, seed=9, species_probs=(0.5, 0.5))
    b = synth.random_box(200, density=0.15, dmin=1.2, seed=9, species_probs=(0.5, 0.5))
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.species, b.species)
    c = synth.random_box(200, density=0.15, dmin=1.2, seed=10)
    assert not np.array_equal(a.pos, c.pos)
