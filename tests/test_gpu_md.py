"""Verlet-skin neighbour-list reuse and velocity-Verlet dynamics around the evaluation.

With a skin the library keeps pairs within r_cut + skin and reuses the list until an atom
has moved by skin/2; pairs beyond r_cut must contribute nothing, so energies and forces equal
those of a fresh list (up to the order of floating-point sums).  The synchronous path with a
fresh list is checked against the oracle in test_gpu_parity.py.
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


def make_model(params, m_sparse=200, zeta=2, skin=0.0, precision="mixed", seed=3):
    from paper_1905_02142_gb300.api import SoapGap
    model = SoapGap.from_dict(params, precision=precision)
    model.set_model(unit_rows(m_sparse, model.dim, seed), synth.gap_weights(m_sparse, seed + 1), zeta)
    model.set_skin(skin)
    return model


def rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def interior_displacement(batch, scale, seed):
    """Random displacements of atoms well inside the cell (fractional 0.1..0.9), so that no
    atom changes image."""
    h = batch.cell[0].reshape(3, 3)
    f = batch.pos @ np.linalg.inv(h)
    inside = np.all((f > 0.1) & (f < 0.9), axis=1)
    d = np.random.default_rng(seed).normal(size=batch.pos.shape)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return batch.pos + scale * d * inside[:, None]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_skin_reuse_matches_fresh_list(precision):
    from paper_1905_02142_gb300.api import Structures
    w = synth.get_workload("box1000_n8l8")
    batch = w.structures()
    skin_model = make_model(w.params(), skin=0.6, precision=precision)
    s = Structures.from_batch(batch)
    tol = 2e-6 if precision == "mixed" else 1e-12
    for step, scale in enumerate([0.0, 0.12, 0.25, 0.45]):
        pos = interior_displacement(batch, scale, seed=step)
        s.pos.copy_(torch.as_tensor(pos, device=s.pos.device))
        got = skin_model.compute(s, energy=True, forces=True, virial=True)
        rebuilt = skin_model.last_rebuild()
        fresh_model = make_model(w.params(), precision=precision)
        ref = fresh_model.compute(Structures(pos, batch.cell, batch.species, batch.atom_offs),
                                  energy=True, forces=True, virial=True)
        # the first call builds; 0.12 and 0.25 A stay below skin / 2 = 0.3 A; 0.45 exceeds it
        assert rebuilt == (1 if scale in (0.0, 0.45) else 0), (scale, rebuilt)
        assert rel(got["forces"], ref["forces"]) < tol
        assert rel(got["e_struct"], ref["e_struct"]) < tol
        assert rel(got["virial"], ref["virial"]) < tol
        fresh_model.close()


def test_skin_reuse_in_captured_graph():
    from paper_1905_02142_gb300.api import CapturedEvaluation, Structures
    w = synth.get_workload("box1000_n8l8")
    batch = w.structures()
    model = make_model(w.params(), skin=0.6)
    s = Structures.from_batch(batch)
    cap = CapturedEvaluation(model, s, energy=True, forces=True)
    for step, scale in enumerate([0.1, 0.2, 0.5, 0.55]):
        pos = interior_displacement(batch, scale, seed=10 + step)
        s.pos.copy_(torch.as_tensor(pos, device=s.pos.device))
        out = cap.replay()
        model.sync_status()
        fresh = make_model(w.params()).compute(Structures(pos, batch.cell, batch.species, batch.atom_offs),
                                               energy=True, forces=True)
        assert rel(out["forces"], fresh["forces"]) < 2e-6, scale
        assert rel(out["e_struct"], fresh["e_struct"]) < 2e-6, scale


def test_velocity_verlet_conserves_energy_and_graph_matches():
    from paper_1905_02142_gb300.api import AMU_A2_PER_FS2_IN_EV, Structures, VelocityVerlet
    box = synth.concat([synth.random_box(512, density=0.1, dmin=1.3, seed=21)])
    params = dict(r_cut=4.5, r_soft=4.0, sigma_r0=0.5, sigma_p0=0.5, n_max=6, l_max=6)
    mass = 12.011
    rng = np.random.default_rng(5)
    kT = 8.617333e-5 * 300.0                       # eV
    vel = rng.normal(size=(512, 3)) * np.sqrt(kT / (mass * AMU_A2_PER_FS2_IN_EV))
    vel -= vel.mean(axis=0)
    runs = {}
    for capture in (False, True):
        model = make_model(params, m_sparse=100, zeta=2, skin=0.5)
        s = Structures.from_batch(box)
        md = VelocityVerlet(model, s, mass, dt=0.5, vel=vel, capture=capture)
        energies = []
        for _ in range(40):
            md.step(5)
            if capture:
                model.sync_status()
            energies.append(md.potential_energy() + md.kinetic_energy())
        runs[capture] = (s.pos.clone(), np.array(energies), md.kinetic_energy())
    pos0, e0, ek = runs[False]
    pos1, e1, _ = runs[True]
    # 200 steps of 0.5 fs: total energy constant to well below the kinetic energy scale
    drift = np.max(np.abs(e0 - e0[0]))
    assert drift < 2e-3 * max(ek, 1.0), (drift, ek)
    # the captured step (device-side list reuse decisions) follows the same trajectory
    np.testing.assert_allclose(e1, e0, rtol=0, atol=1e-9 * max(1.0, abs(e0[0])))
    assert torch.allclose(pos1, pos0, rtol=0, atol=1e-10)


# ------------------------------------------------------------------ against the oracle
def wrapped(pos, cell):
    """Positions mapped into the cell (fractional coordinates modulo 1): the same periodic
    structure, in the form the oracle's neighbour search takes."""
    h = np.asarray(cell).reshape(3, 3)
    f = pos @ np.linalg.inv(h)
    f -= np.floor(f)
    f[f >= 1.0] = 0.0
    return f @ h


def oracle_check(batch_now, P, qs, al, zeta, got, atoms, tol_e, tol_f, label):
    """Local energies and forces of sampled atoms against the oracle at the current positions."""
    from oracle import gap, soap
    from parity_helpers import oracle_W, rel_all
    W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
    fr, atoms = gap.forces_at(batch_now, P, qs, al, zeta, atoms, W=W)
    d = soap.descriptors(batch_now, P, centers=atoms, W=W)
    eps = gap.local_energies(d["q"], torch.as_tensor(qs), torch.as_tensor(al), zeta).numpy()
    e_err = rel_all(got["e_atom"].double().cpu().numpy()[atoms][None], eps[None])
    f_err = rel_all(got["forces"].cpu().numpy()[atoms], fr)
    print(f"PARITY {label}: eps {e_err:.2e} F {f_err:.2e}")
    assert e_err < tol_e and f_err < tol_f


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_skin_reuse_against_oracle(precision):
    """After two reuse steps of a skin list (atoms moved by 0.12 and then 0.25 A, below
    skin / 2), sampled energies and forces equal the oracle's at the moved positions."""
    from oracle import Params
    from paper_1905_02142_gb300.api import SoapGap, Structures
    from parity_helpers import sparse_model
    w = synth.get_workload("box1000_n8l8")
    batch = w.structures()
    P, qs, al, zeta = sparse_model("box1000_n8l8", 100)
    model = SoapGap.from_dict(w.params(), precision=precision)
    model.set_model(qs, al, zeta)
    model.set_skin(0.6)
    s = Structures.from_batch(batch)
    model.compute(s, energy=True, forces=True)
    assert model.last_rebuild() == 1
    for step, scale in enumerate([0.12, 0.25]):
        pos = interior_displacement(batch, scale, seed=step + 1)
        s.pos.copy_(torch.as_tensor(pos, device=s.pos.device))
        got = model.compute(s, energy=True, forces=True)
        assert model.last_rebuild() == 0
    now = synth.Batch(pos, batch.cell, batch.species, batch.atom_offs)
    atoms = np.random.default_rng(31).choice(batch.n_atoms, 6, replace=False)
    tol = (1e-4, 1e-3) if precision == "mixed" else (1e-10, 1e-9)
    oracle_check(now, Params.from_dict(w.params()), qs, al, zeta, got, atoms, *tol,
                 f"skin reuse box1000 {precision}")


def test_captured_md_against_oracle():
    """Forty velocity-Verlet steps replayed from a captured graph with a Verlet skin: the
    structure energy and all forces of the final state equal the oracle's at the final
    positions (unwrapped on the device, mapped into the cell for the oracle)."""
    from oracle import Params, gap, soap
    from paper_1905_02142_gb300.api import AMU_A2_PER_FS2_IN_EV, SoapGap, Structures, VelocityVerlet
    from parity_helpers import oracle_W
    box = synth.concat([synth.random_box(512, density=0.1, dmin=1.3, seed=21)])
    params = dict(r_cut=4.5, r_soft=4.0, sigma_r0=0.5, sigma_p0=0.5, n_max=6, l_max=6)
    P = Params(**params)
    W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
    sparse_box = synth.concat([synth.random_box(60, density=0.1, dmin=1.3, seed=22)])
    qs = soap.descriptors(sparse_box, P, W=W)["q"].numpy()
    al = synth.gap_weights(len(qs), 23)
    model = SoapGap.from_dict(params, precision="mixed")
    model.set_model(qs, al, 2.0)
    model.set_skin(0.5)
    mass = 12.011
    kT = 8.617333e-5 * 600.0
    vel = np.random.default_rng(6).normal(size=(512, 3)) * np.sqrt(kT / (mass * AMU_A2_PER_FS2_IN_EV))
    vel -= vel.mean(axis=0)
    s = Structures.from_batch(box)
    md = VelocityVerlet(model, s, mass, dt=1.0, vel=vel, capture=True)
    md.step(40)
    model.sync_status()
    torch.cuda.synchronize()
    pos = wrapped(s.pos.cpu().numpy(), box.cell[0])
    now = synth.Batch(pos, box.cell, box.species, box.atom_offs)
    moved = np.linalg.norm(s.pos.cpu().numpy() - box.pos, axis=1).max()
    assert moved > 0.05                      # the atoms did move
    ref = gap.evaluate(now, P, qs, al, 2.0, W=W, virial=False)
    e_err = abs(md.potential_energy() - ref["e_struct"].sum()) / abs(ref["e_struct"].sum())
    f_err = np.linalg.norm(md.f.cpu().numpy() - ref["forces"]) / np.linalg.norm(ref["forces"])
    print(f"PARITY captured MD 40 steps: E {e_err:.2e} F {f_err:.2e} (max displacement {moved:.2f} A)")
    assert e_err < 1e-4 and f_err < 1e-3
