"""Asynchronous (graph-capturable) evaluation and the autotuner.

A CUDA graph captured from an asynchronous soapgap_compute call must reproduce the
synchronous call exactly, follow positions changed in place between replays, and report a
pair-buffer overflow through soapgap_sync_status instead of writing past the buffers.
The synchronous path itself is checked against the oracle in test_gpu_parity.py.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_02142_gb300 import build
    build.build()


def unit_rows(m, d, seed):
    rng = np.random.default_rng(seed)
    q = np.abs(rng.normal(size=(m, d)))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def make_model(params, m_sparse, zeta, seed=3):
    from paper_1905_02142_gb300.api import SoapGap
    model = SoapGap.from_dict(params, precision="mixed")
    model.set_model(unit_rows(m_sparse, model.dim, seed), synth.gap_weights(m_sparse, seed + 1), zeta)
    return model


OUT = dict(energy=True, forces=True, virial=True)


def rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


def wrap_into_cells(pos, cell, offs):
    """Positions mapped back into their cells (fractional coordinates modulo 1)."""
    out = pos.copy()
    for s in range(len(offs) - 1):
        a, b = offs[s], offs[s + 1]
        h = cell[s].reshape(3, 3)
        f = out[a:b] @ np.linalg.inv(h)
        f -= np.floor(f)
        f[f >= 1.0] = 0.0
        out[a:b] = f @ h
    return out


@pytest.fixture(scope="module")
def batched():
    w = synth.get_workload("batch256_n8l8")
    return w, w.structures()


def test_captured_graph_matches_synchronous_call(batched):
    from paper_1905_02142_gb300.api import CapturedEvaluation, Structures
    w, batch = batched
    model = make_model(w.params(), w.n_sparse, w.zeta)
    s = Structures.from_batch(batch)
    ref = model.compute(s, **OUT)
    ref = {k: v.clone() for k, v in ref.items()}
    cap = CapturedEvaluation(model, s, **OUT)
    for _ in range(2):
        out = cap.replay()
    model.sync_status()
    for k in ("e_struct", "forces", "e_atom"):
        assert torch.equal(out[k], ref[k]), k
    assert torch.allclose(out["virial"], ref["virial"], rtol=1e-12, atol=0)


def test_replay_follows_positions_changed_in_place(batched):
    from paper_1905_02142_gb300.api import CapturedEvaluation, Structures
    w, batch = batched
    model = make_model(w.params(), w.n_sparse, w.zeta)
    s = Structures.from_batch(batch)
    cap = CapturedEvaluation(model, s, **OUT)
    rng = np.random.default_rng(9)
    moved = wrap_into_cells(batch.pos + 0.03 * rng.normal(size=batch.pos.shape), batch.cell,
                            batch.atom_offs)
    s.pos.copy_(torch.as_tensor(moved, device=s.pos.device))
    out = cap.replay()
    model.sync_status()
    fresh_model = make_model(w.params(), w.n_sparse, w.zeta)
    fresh = fresh_model.compute(Structures(moved, batch.cell, batch.species, batch.atom_offs), **OUT)
    assert torch.equal(out["forces"], fresh["forces"])
    assert torch.equal(out["e_struct"], fresh["e_struct"])
    assert torch.allclose(out["virial"], fresh["virial"], rtol=1e-6, atol=1e-9)


def test_pair_overflow_reported_not_written():
    from paper_1905_02142_gb300.api import CapturedEvaluation, SoapGapError, Structures
    from paper_1905_02142_gb300 import _lib as L
    w = synth.get_workload("box1000_n8l8")
    batch = w.structures()
    model = make_model(w.params(), 200, 2)
    s = Structures.from_batch(batch)
    cap = CapturedEvaluation(model, s, **OUT)
    first = {k: v.clone() for k, v in cap.replay().items()}
    model.sync_status()
    # squeeze the atoms towards the cell origin: about twice the pairs of the capture
    s.pos.mul_(0.8)
    cap.replay()
    with pytest.raises(SoapGapError) as err:
        model.sync_status()
    assert err.value.code == L.E_CAPACITY
    s.pos.copy_(torch.as_tensor(batch.pos, device=s.pos.device))
    again = cap.replay()
    model.sync_status()
    for k in ("e_struct", "forces"):
        assert torch.equal(again[k], first[k]), k


def test_async_call_needs_sized_workspace():
    from paper_1905_02142_gb300.api import SoapGapError, Structures
    from paper_1905_02142_gb300 import _lib as L
    w = synth.get_workload("box64_n6l6")
    model = make_model(w.params(), 50, 2)
    with pytest.raises(SoapGapError) as err:
        model.compute(Structures.from_batch(w.structures()), asynchronous=True, **OUT)
    assert err.value.code == L.E_STATE


def test_autotune_keeps_results(batched):
    from paper_1905_02142_gb300.api import Structures
    w, batch = batched
    model = make_model(w.params(), w.n_sparse, w.zeta)
    s = Structures.from_batch(batch)
    before = {k: v.clone() for k, v in model.compute(s, **OUT).items()}
    plan = model.autotune(s)
    assert plan["adjoint_warps"] in (2, 3, 4, 5)
    assert 0 <= plan["gap_forward"] < 3 and 0 <= plan["gap_backward"] < 5
    assert plan["pair_forward"] in (1, 2)
    assert model.plan(s) == {k: plan[k] for k in model.PLAN_KEYS}
    after = model.compute(s, **OUT)
    # results depend on the plan only through the order of floating-point sums
    for k in ("forces", "e_struct", "virial"):
        assert rel(after[k], before[k]) < 1e-5, k


def test_every_tile_plan_gives_the_same_results(batched):
    """All GEMM tile configurations of the GAP products, adjoint block shapes and neighbour
    sweeps give the same energies and forces, up to the order of sums, for each forward
    kernel; the two forward kernels agree to their precision."""
    import itertools

    from paper_1905_02142_gb300.api import SoapGapError, Structures
    from paper_1905_02142_gb300 import _lib as L
    w, batch = batched
    model = make_model(w.params(), w.n_sparse, w.zeta)
    s = Structures.from_batch(batch)
    model.compute(s, **OUT)
    assert model.plan(s) == {"adjoint_warps": 0, "gap_forward": 0, "gap_backward": 0, "neighbour_sweep": 0,
                             "pair_forward": 0}
    base = {"adjoint_warps": 0, "gap_forward": 0, "gap_backward": 0, "neighbour_sweep": 0}
    ref = {}
    for pf in (1, 2):  # the two forward kernels differ in arithmetic, not only in the order of sums
        model.set_plan(s, dict(base, pair_forward=pf))
        ref[pf] = {k: v.clone() for k, v in model.compute(s, **OUT).items()}
    for k, bar in (("forces", 1e-4), ("e_struct", 1e-5), ("e_atom", 1e-4)):
        assert rel(ref[2][k], ref[1][k]) < bar, (k, rel(ref[2][k], ref[1][k]))
    for warps, fwd, bwd in itertools.product((2, 4, 5), range(3), range(5)):
        pf = 1 + (fwd + 2 * bwd + warps) % 2
        model.set_plan(s, {"adjoint_warps": warps, "gap_forward": fwd, "gap_backward": bwd,
                           "neighbour_sweep": (fwd + bwd) % 3, "pair_forward": pf})
        out = model.compute(s, **OUT)
        # norm-wise: the local energies are sums of terms far larger than themselves, so
        # their last bits follow the partial-sum layout of the forward tile shape
        for k, bar in (("forces", 1e-5), ("e_struct", 1e-5), ("e_atom", 5e-5)):
            assert rel(out[k], ref[pf][k]) < bar, (k, warps, fwd, bwd, pf, rel(out[k], ref[pf][k]))
    with pytest.raises(SoapGapError) as err:
        model.set_plan(s, {"adjoint_warps": 6, "gap_forward": 0, "gap_backward": 0, "neighbour_sweep": 0,
                           "pair_forward": 0})
    with pytest.raises(SoapGapError) as err:
        model.set_plan(s, {"adjoint_warps": 0, "gap_forward": 0, "gap_backward": 0, "neighbour_sweep": 0,
                           "pair_forward": 3})
    assert err.value.code == L.E_INVALID_ARG


def test_plan_cache_round_trip(batched, tmp_path):
    from paper_1905_02142_gb300.api import Structures
    w, batch = batched
    cache = str(tmp_path / "plans.json")
    model = make_model(w.params(), w.n_sparse, w.zeta)
    s = Structures.from_batch(batch)
    first = model.autotune(s, cache=cache)
    assert not first["cached"]
    other = make_model(w.params(), w.n_sparse, w.zeta)
    second = other.autotune(s, cache=cache)
    assert second["cached"]
    assert {k: second[k] for k in other.PLAN_KEYS} == {k: first[k] for k in model.PLAN_KEYS}
    assert other.plan(s) == {k: first[k] for k in model.PLAN_KEYS}


def test_plan_cache_entry_without_the_forward_kernel_is_retuned(batched, tmp_path):
    """A cache entry written before the plan held the forward-kernel choice is timed again
    and replaced, not read with a missing key."""
    import json

    from paper_1905_02142_gb300.api import Structures
    w, batch = batched
    cache = str(tmp_path / "plans.json")
    model = make_model(w.params(), w.n_sparse, w.zeta)
    s = Structures.from_batch(batch)
    model.autotune(s, cache=cache)
    with open(cache) as f:
        known = json.load(f)
    for entry in known.values():
        entry.pop("pair_forward")
    with open(cache, "w") as f:
        json.dump(known, f)
    other = make_model(w.params(), w.n_sparse, w.zeta)
    again = other.autotune(s, cache=cache)
    assert not again["cached"]
    with open(cache) as f:
        assert all("pair_forward" in e for e in json.load(f).values())
