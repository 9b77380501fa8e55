"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

Bars (relative, see parity_helpers):
  neighbour pairs   bit-exact (same (i, j, S) list in canonical order)
  FP64 path         p within 1e-11 where cond(S) allows (n_max <= 6), else within
                    4 eps sqrt(cond S); energies max(1e-10, 0.1 eps sqrt(cond S)); forces
                    max(1e-9, 2 eps sqrt(cond S)) (see fp64_tols)
  mixed path        p within 1e-5; energies 1e-4; forces 1e-3 RMS
"""
import numpy as np
import pytest
import torch

import synth
from oracle import Params, basis, gap, neighbours, soap

from parity_helpers import oracle_W, rel_all, rel_rows, sparse_model

pytestmark = pytest.mark.gpu

MIXED = dict(p=1e-5, e=1e-4, f=1e-3)


def rounding_scale(P):
    """eps sqrt(cond S): the relative rounding that W = S^-1/2 carries into b_n = W b_alpha
    from an O(eps) error in the primitive radial integrals (Sec. III.A; cond S grows from
    ~1e9 at n_max = 6 to ~6e16 at n_max = 12)."""
    cond = np.linalg.cond(basis.overlap_matrix(P.n_max, P.r_cut, P.sigma_r0))
    return 2.2e-16 * np.sqrt(cond)


def fp64_p_tol(P):
    """p bar of the FP64 path: 1e-11 where the basis allows it, else 4 eps sqrt(cond S).
    Measured on GB300 against the oracle, in units of r = eps sqrt(cond S): 0.3 r (n_max 6),
    0.5-0.6 r (n_max 8), 0.45 r (n_max 10, the benchmark box), 1.5 r (n_max 12)."""
    return max(1e-11, 4 * rounding_scale(P))


def fp64_tols(P):
    """Bars of the FP64 path: p; energies max(1e-10, 0.1 r) (measured at most 0.016 r, at
    n_max 10); forces max(1e-9, 2 r) (measured at most 0.8 r, at n_max 10)."""
    r = rounding_scale(P)
    return dict(p=fp64_p_tol(P), e=max(1e-10, 0.1 * r), f=max(1e-9, 2 * r))


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_02142_gb300 import build
    build.build()


def model_for(params: dict, precision, qs=None, al=None, zeta=None):
    from paper_1905_02142_gb300.api import SoapGap
    m = SoapGap.from_dict(params, precision=precision)
    if qs is not None:
        m.set_model(qs, al, zeta)
    return m


def structures(batch):
    from paper_1905_02142_gb300.api import Structures
    return Structures.from_batch(batch)


def params_dict(P: Params):
    return dict(r_cut=P.r_cut, r_soft=P.r_soft, sigma_r0=P.sigma_r0, sigma_p0=P.sigma_p0,
                alpha_r=P.alpha_r, alpha_p=P.alpha_p, amp_a=P.amp_a, n_f=P.n_f,
                central_weight=P.central_weight, n_max=P.n_max, l_max=P.l_max,
                n_species=P.n_species, eq08_weight=P.eq08_weight)


def oracle_pairs(batch, r_cut, centers=None):
    pr = neighbours.batch_pairs(batch, r_cut, centers=centers)
    return pr["i"], pr["j"], pr["shift"]


# ------------------------------------------------------------------ neighbours
SMALL_BATCH = synth.batched_boxes(10, n_lo=4, n_hi=150, seed=77)


@pytest.mark.parametrize("sweep", [1, 2])
@pytest.mark.parametrize("case", ["box64_n6l6", "box1000_n8l8", "twospecies4096_n8l8", "batch",
                                  "triclinic_small"])
def test_pair_list_bit_exact(case, sweep):
    """Both candidate sweeps (per bin from staged shared memory, per atom) give the oracle's
    pair list exactly."""
    if case == "batch":
        batch, P = SMALL_BATCH, Params(r_cut=4.5, r_soft=4.0, sigma_r0=0.5, sigma_p0=0.5)
    elif case == "triclinic_small":
        batch = synth.concat([synth.random_box(7, side=3.1, dmin=1.0, seed=5, shear=0.35,
                                               species_probs=(0.5, 0.5))])
        P = Params(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, n_species=2)
    else:
        w = synth.get_workload(case)
        batch, P = w.structures(), Params.from_dict(w.params())
    m = model_for(params_dict(P), "mixed")
    s = structures(batch)
    m.compute(s, desc=True)
    m.set_plan(s, {"adjoint_warps": 0, "gap_forward": 0, "gap_backward": 0, "neighbour_sweep": sweep,
                   "pair_forward": 0})
    m.compute(s, desc=True)
    gi, gj, gs = m.pairs()
    oi, oj, os_ = oracle_pairs(batch, P.r_cut)
    assert len(gi) == len(oi)
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj) and np.array_equal(gs, os_)


def test_pair_list_bit_exact_100k_sampled():
    w = synth.get_workload("box100k_n10l10")
    batch = w.structures()
    m = model_for(w.params(), "mixed")
    m.compute(structures(batch), desc=True)
    gi, gj, gs = m.pairs()
    centers = np.sort(np.random.default_rng(0).choice(batch.n_atoms, 24, replace=False))
    oi, oj, os_ = oracle_pairs(batch, w.r_cut, centers=centers)
    sel = np.isin(gi, centers)
    assert np.array_equal(gi[sel], oi) and np.array_equal(gj[sel], oj) and np.array_equal(gs[sel], os_)
    # every pair has its reverse (symmetry) and the count matches the density estimate
    assert len(gi) == pytest.approx(batch.n_atoms * 0.15 * 4 / 3 * np.pi * 125, rel=0.05)


# ------------------------------------------------------------------ descriptors
@pytest.mark.parametrize("name,precision", [("box64_n6l6", "fp64"), ("box64_n6l6", "mixed"),
                                            ("box1000_n8l8", "fp64"), ("box1000_n8l8", "mixed")])
def test_descriptors(name, precision):
    w = synth.get_workload(name)
    batch, P = w.structures(), Params.from_dict(w.params())
    m = model_for(w.params(), precision)
    out = m.compute(structures(batch), desc=True)
    q = out["q"].double().cpu().numpy()
    pn = out["pnorm"].double().cpu().numpy()
    centers = None if batch.n_atoms <= 1000 else np.arange(0, batch.n_atoms, 7)
    ref = soap.descriptors(batch, P, centers=centers, W=oracle_W(P.n_max, P.r_cut, P.sigma_r0))
    c = ref["centers"]
    p_gpu = q[c] * pn[c][:, None]
    p_ref = (ref["q"] * ref["pnorm"][:, None]).numpy()
    err = rel_rows(p_gpu, p_ref)
    tol = fp64_p_tol(P) if precision == "fp64" else MIXED["p"]
    print(f"PARITY {name} {precision}: max rel err of p = {err:.3e} (tol {tol:.1e})")
    assert err < tol


# ------------------------------------------------------------------ energies and forces
def check_energy_forces(batch, name, precision, m_sparse=None, atoms_for_forces=None, virial=True,
                        desc=False):
    P, qs, al, zeta = sparse_model(name, m_sparse)
    model = model_for(params_dict(P), precision, qs, al, zeta)
    out = model.compute(structures(batch), desc=desc, energy=True, forces=True, virial=virial)
    e_atom = out["e_atom"].double().cpu().numpy()
    e_struct = out["e_struct"].cpu().numpy()
    f = out["forces"].cpu().numpy()
    W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
    tol = MIXED if precision == "mixed" else fp64_tols(P)
    if atoms_for_forces is None:
        ref = gap.evaluate(batch, P, qs, al, zeta, W=W, virial=virial)
        e_err = rel_all(e_atom[None], ref["e_atom"][None])
        es_err = float(np.max(np.abs(e_struct - ref["e_struct"]) / np.abs(ref["e_struct"])))
        f_err = rel_all(f, ref["forces"])
        v_err = rel_all(out["virial"].cpu().numpy().reshape(-1, 9),
                        ref["virial"].reshape(-1, 9)) if virial else 0.0
    else:
        fr, atoms = gap.forces_at(batch, P, qs, al, zeta, atoms_for_forces, W=W)
        d = soap.descriptors(batch, P, centers=atoms, W=W)
        eps = gap.local_energies(d["q"], torch.as_tensor(qs), torch.as_tensor(al), zeta).numpy()
        e_err = rel_all(e_atom[atoms][None], eps[None])
        es_err = 0.0
        f_err = rel_all(f[atoms], fr)
        v_err = 0.0
    print(f"PARITY {name} {precision}: eps {e_err:.2e} E {es_err:.2e} F {f_err:.2e} W {v_err:.2e} "
          f"(bars e {tol['e']:.1e} f {tol['f']:.1e})")
    assert e_err < tol["e"] and es_err < tol["e"]
    assert f_err < tol["f"] and v_err < tol["f"]
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_forces_box64(precision):
    w = synth.get_workload("box64_n6l6")
    check_energy_forces(w.structures(), "box64_n6l6", precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_forces_box1000(precision):
    w = synth.get_workload("box1000_n8l8")
    check_energy_forces(w.structures(), "box1000_n8l8", precision, m_sparse=100)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_forces_small_batch(precision):
    check_energy_forces(SMALL_BATCH, "batch256_n8l8", precision, m_sparse=64)


def sampled_p_error(batch, P, out, centers):
    """Max relative error of p = q |p| over the listed centres against the oracle."""
    q = out["q"].double().cpu().numpy()
    pn = out["pnorm"].double().cpu().numpy()
    ref = soap.descriptors(batch, P, centers=np.sort(centers), W=oracle_W(P.n_max, P.r_cut, P.sigma_r0))
    c = ref["centers"]
    return rel_rows(q[c] * pn[c][:, None], (ref["q"] * ref["pnorm"][:, None]).numpy())


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_energy_forces_two_species_sampled(precision):
    w = synth.get_workload("twospecies4096_n8l8")
    P = Params.from_dict(w.params())
    atoms = np.random.default_rng(1).choice(4096, 6, replace=False)
    out = check_energy_forces(w.structures(), "twospecies4096_n8l8", precision, m_sparse=300,
                              atoms_for_forces=atoms, virial=False, desc=True)
    err = sampled_p_error(w.structures(), P, out, np.random.default_rng(11).choice(4096, 16, replace=False))
    tol = MIXED["p"] if precision == "mixed" else fp64_p_tol(P)
    print(f"PARITY twospecies4096_n8l8 {precision}: sampled p {err:.3e} (tol {tol:.1e})")
    assert err < tol


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_energy_forces_100k_sampled_full_model(precision):
    """The bench workload (100 000 atoms, n = l = 10, 4000 sparse environments, zeta 4) in
    the launch configuration the benchmark times, on both paths: p of 16 sampled centres,
    local energies and forces of 4 sampled atoms against the oracle."""
    w = synth.get_workload("box100k_n10l10")
    P = Params.from_dict(w.params())
    atoms = np.random.default_rng(2).choice(w.n_atoms, 4, replace=False)
    out = check_energy_forces(w.structures(), "box100k_n10l10", precision, atoms_for_forces=atoms,
                              virial=False, desc=True)
    err = sampled_p_error(w.structures(), P, out,
                          np.random.default_rng(12).choice(w.n_atoms, 16, replace=False))
    tol = MIXED["p"] if precision == "mixed" else fp64_p_tol(P)
    print(f"PARITY box100k_n10l10 {precision}: sampled p {err:.3e} (tol {tol:.1e})")
    assert err < tol


# the corners of the paper's timing grid (Sec. III.D: 10 000 atoms in a 46.371 A cube, no two
# closer than 0.7 A; r_cut 5 A and sigma 0.5 A, which the paper does not state)
TIMING_BOX = synth.concat([synth.random_box(10000, side=46.371, dmin=0.7, seed=2019)])


@pytest.mark.parametrize("n_max,l_max,precision", [(3, 3, "mixed"), (12, 12, "mixed"), (11, 12, "mixed"),
                                                   (12, 3, "mixed"), (3, 3, "fp64"), (12, 12, "fp64")])
def test_timing_grid_corners(n_max, l_max, precision):
    P = Params(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, n_max=n_max, l_max=l_max)
    m = model_for(params_dict(P), precision)
    out = m.compute(structures(TIMING_BOX), desc=True)
    centers = np.random.default_rng(n_max * 100 + l_max).choice(TIMING_BOX.n_atoms, 12, replace=False)
    err = sampled_p_error(TIMING_BOX, P, out, centers)
    tol = MIXED["p"] if precision == "mixed" else fp64_p_tol(P)
    print(f"PARITY timing box n={n_max} l={l_max} {precision}: sampled p {err:.3e} (tol {tol:.1e})")
    assert err < tol


# ------------------------------------------------------------------ hyperparameter variants
def hp_variants(golden):
    hs = golden["hyperparameter_sets"]
    out = []
    for key in ("optimised_adsorption_informed", "sobol_optimum", "fair_comparison"):
        h = hs[key]
        out.append(Params(r_cut=h["r_cut"], r_soft=h["r_cut"] - 0.5, sigma_r0=h["sigma_r0"],
                          sigma_p0=h["sigma_p0"], alpha_r=h["alpha_r"], alpha_p=h["alpha_p"],
                          amp_a=h["amp_a"], n_max=h["n_max"], l_max=h["l_max"]))
    out.append(Params(r_cut=4.0, r_soft=4.0, sigma_r0=0.5, sigma_p0=0.5, n_max=2, l_max=0))
    out.append(Params(r_cut=4.0, r_soft=3.0, sigma_r0=0.4, sigma_p0=0.6, n_max=5, l_max=11,
                      eq08_weight=True, central_weight=0.0))
    return out


@pytest.mark.parametrize("k", range(5))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hyperparameter_variants(golden, k, precision):
    P = hp_variants(golden)[k]
    batch = synth.concat([synth.random_box(40, side=7.5, dmin=1.0, seed=40 + k)])
    W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
    qs = soap.descriptors(synth.concat([synth.random_box(12, side=5.0, dmin=1.0, seed=90 + k)]),
                          P, W=W)["q"].numpy()
    al = synth.gap_weights(len(qs), 5 + k)
    zeta = 3.0 if k < 2 else 2.0
    model = model_for(params_dict(P), precision, qs, al, zeta)
    out = model.compute(structures(batch), desc=True, energy=True, forces=True)
    ref_d = soap.descriptors(batch, P, W=W)
    ref = gap.evaluate(batch, P, qs, al, zeta, W=W, virial=False)
    p_gpu = out["q"].double().cpu().numpy() * out["pnorm"].double().cpu().numpy()[:, None]
    p_err = rel_rows(p_gpu, (ref_d["q"] * ref_d["pnorm"][:, None]).numpy())
    e_err = rel_all(out["e_atom"].double().cpu().numpy()[None], ref["e_atom"][None])
    f_err = rel_all(out["forces"].cpu().numpy(), ref["forces"])
    terms = model.gap_terms()[0] if precision == "mixed" else 0
    print(f"PARITY HP set {k} {precision}: p {p_err:.2e} eps {e_err:.2e} F {f_err:.2e} "
          f"(GAP products {terms})")
    if precision == "mixed":
        assert p_err < MIXED["p"] and e_err < MIXED["e"] and f_err < MIXED["f"]
    else:
        tol = fp64_tols(P)
        assert p_err < tol["p"] and e_err < tol["e"] and f_err < tol["f"]


# ------------------------------------------------------------------ API paths and edges
def test_autograd_function_matches_forces():
    from paper_1905_02142_gb300.api import SoapGapEnergy
    P, qs, al, zeta = sparse_model("box64_n6l6")
    batch = SMALL_BATCH
    model = model_for(params_dict(P), "fp64", qs, al, zeta)
    s = structures(batch)
    out = model.compute(s, energy=True, forces=True)
    pos = s.pos.clone().requires_grad_(True)
    w = torch.linspace(0.5, 2.0, s.n_struct, dtype=torch.float64, device=pos.device)
    e = SoapGapEnergy.apply(pos, model, s)
    (e * w).sum().backward()
    atom_w = torch.repeat_interleave(w, torch.as_tensor(np.diff(batch.atom_offs), device=pos.device))
    assert torch.allclose(pos.grad, -out["forces"] * atom_w[:, None], rtol=1e-10, atol=1e-12)
    assert torch.allclose(e, out["e_struct"], rtol=1e-12)


def test_backward_matches_central_differences_fp64():
    P, qs, al, zeta = sparse_model("box64_n6l6")
    batch = synth.concat([synth.random_box(20, side=5.5, dmin=1.2, seed=21, shear=0.1)])
    model = model_for(params_dict(P), "fp64", qs, al, zeta)
    s = structures(batch)
    out = model.compute(s, energy=True, forces=True)
    f = out["forces"].cpu().numpy()
    h = 1e-5
    for atom, comp in [(0, 0), (5, 2), (13, 1)]:
        vals = []
        for sgn in (1, -1):
            pos = batch.pos.copy()
            pos[atom, comp] += sgn * h
            b2 = synth.Batch(pos, batch.cell, batch.species, batch.atom_offs)
            vals.append(float(model.compute(structures(b2), energy=True)["e_struct"].sum()))
        fd = -(vals[0] - vals[1]) / (2 * h)
        assert f[atom, comp] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_compute_host_matches_device():
    P, qs, al, zeta = sparse_model("box64_n6l6")
    batch = SMALL_BATCH
    model = model_for(params_dict(P), "mixed", qs, al, zeta)
    dev = model.compute(structures(batch), desc=True, energy=True, forces=True, virial=True)
    host = model.compute_host(batch.pos, batch.cell, batch.species, batch.atom_offs, desc=True,
                              energy=True, forces=True, virial=True)
    for k in ("q", "e_struct", "forces", "virial"):
        assert np.array_equal(dev[k].cpu().numpy(), host[k]), k


def test_empty_structures_and_isolated_atoms():
    P, qs, al, zeta = sparse_model("box64_n6l6")
    lone = synth.Structure(pos=np.array([[5.0, 5.0, 5.0]]), cell=np.eye(3) * 20.0,
                           species=np.zeros(1, np.int32))
    empty = synth.Structure(pos=np.zeros((0, 3)), cell=np.eye(3) * 9.0, species=np.zeros(0, np.int32))
    box = synth.random_box(16, side=5.0, dmin=1.2, seed=3)
    batch = synth.concat([empty, lone, box, empty])
    model = model_for(params_dict(P), "fp64", qs, al, zeta)
    out = model.compute(structures(batch), desc=True, energy=True, forces=True, virial=True)
    ref = gap.evaluate(batch, P, qs, al, zeta, W=oracle_W(P.n_max, P.r_cut, P.sigma_r0))
    assert np.allclose(out["e_struct"].cpu().numpy(), ref["e_struct"], rtol=1e-10, atol=1e-14)
    assert np.allclose(out["forces"].cpu().numpy(), ref["forces"], rtol=1e-8, atol=1e-12)
    assert float(out["e_struct"][0]) == 0.0 and float(out["e_struct"][3]) == 0.0
    assert np.all(out["forces"][0].cpu().numpy() == 0.0)


def test_invalid_inputs_are_reported():
    from paper_1905_02142_gb300.api import SoapGapError
    P, qs, al, zeta = sparse_model("box64_n6l6")
    model = model_for(params_dict(P), "mixed", qs, al, zeta)
    # an atom displaced by lattice vectors is the same structure (mapped into its cell)
    inside = synth.random_box(20, side=8.0, dmin=1.2, seed=12)
    shifted = synth.Structure(pos=inside.pos + np.array([[8.0, -16.0, 0.0]] * 3 + [[0.0, 0.0, 0.0]] * 17),
                              cell=inside.cell, species=inside.species)
    a = model.compute(structures(synth.concat([inside])), energy=True, forces=True)
    b = model.compute(structures(synth.concat([shifted])), energy=True, forces=True)
    assert torch.allclose(a["e_struct"], b["e_struct"], rtol=1e-6, atol=0)
    assert torch.allclose(a["forces"], b["forces"], rtol=0, atol=1e-6 * float(a["forces"].abs().max()))
    bad = synth.Structure(pos=np.array([[1.0, 1.0, 1.0], [np.nan, 1.0, 1.0]]), cell=np.eye(3) * 8.0,
                          species=np.zeros(2, np.int32))
    with pytest.raises(SoapGapError) as e:
        model.compute(structures(synth.concat([bad])), desc=True)
    assert "not finite" in str(e.value)
    same = synth.Structure(pos=np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0]]), cell=np.eye(3) * 8.0,
                           species=np.zeros(2, np.int32))
    with pytest.raises(SoapGapError) as e:
        model.compute(structures(synth.concat([same])), desc=True)
    assert "coincide" in str(e.value)
    # the handle stays usable after an error
    ok = model.compute(structures(synth.concat([synth.random_box(8, side=5.0, seed=1)])), energy=True)
    assert torch.isfinite(ok["e_struct"]).all()


def test_model_replacement_and_invalid_models():
    """An invalid model is refused and leaves the previous one in place; a replaced model
    needs a new energy evaluation before the adjoint."""
    from paper_1905_02142_gb300 import _lib as L
    from paper_1905_02142_gb300.api import SoapGapError
    P, qs, al, zeta = sparse_model("box64_n6l6")
    model = model_for(params_dict(P), "mixed", qs, al, zeta)
    s = structures(SMALL_BATCH)
    e0 = model.compute(s, energy=True)["e_struct"].clone()
    bad = np.array(al, dtype=np.float64)
    bad[3] = np.nan
    with pytest.raises(SoapGapError) as e:
        model.set_model(qs, bad, zeta)
    assert e.value.code == L.E_INVALID_ARG
    assert torch.equal(model.compute(s, energy=True)["e_struct"], e0)
    model.set_model(qs, 2 * np.asarray(al), zeta)
    w = torch.ones(s.n_struct, dtype=torch.float64, device=e0.device)
    with pytest.raises(SoapGapError) as e:
        model.backward(s, w)
    assert e.value.code == L.E_STATE
    e1 = model.compute(s, energy=True)["e_struct"]
    scale = float(e0.abs().max())
    assert torch.allclose(e1, 2 * e0, rtol=1e-5, atol=1e-5 * scale)
    assert torch.isfinite(model.backward(s, w)).all()


def test_failed_evaluation_leaves_no_forward_for_the_adjoint():
    """A call that fails part-way has rewritten the workspace: the adjoint of the last
    successful evaluation of the same batch shape is refused until a new one succeeds."""
    from paper_1905_02142_gb300 import _lib as L
    from paper_1905_02142_gb300.api import SoapGapError
    P, qs, al, zeta = sparse_model("box64_n6l6")
    model = model_for(params_dict(P), "mixed", qs, al, zeta)
    good = synth.random_box(20, side=8.0, dmin=1.2, seed=12)
    pos = good.pos.copy()
    pos[1] = pos[0]                                   # same shape, two atoms coincide
    bad = synth.Structure(pos=pos, cell=good.cell, species=good.species)
    s_good = structures(synth.concat([good]))
    w = torch.ones(1, dtype=torch.float64, device=s_good.pos.device)
    model.compute(s_good, energy=True)
    g0 = model.backward(s_good, w)
    with pytest.raises(SoapGapError) as e:
        model.compute(structures(synth.concat([bad])), energy=True)
    assert "coincide" in str(e.value)
    with pytest.raises(SoapGapError) as e:
        model.backward(s_good, w)
    assert e.value.code == L.E_STATE
    model.compute(s_good, energy=True)
    assert torch.equal(model.backward(s_good, w), g0)


@pytest.mark.parametrize("sweep", [1, 2])
def test_pair_list_dense_corner_cluster(sweep):
    """Atoms squeezed into one corner of a large cell: far more neighbours per atom than the
    cell's mean density predicts, so the library's first neighbour sweep overflows its
    per-atom slots and is redone with the measured count.  The pair list must still equal
    the oracle's exactly."""
    base = synth.random_box(300, density=0.15, dmin=1.2, seed=41)
    batch = synth.concat([base])
    batch.pos[:] = batch.pos * 0.55          # same cell, 6x the local density
    P = Params(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, n_max=6, l_max=6)
    m = model_for(params_dict(P), "mixed")
    s = structures(batch)
    m.compute(s, desc=True)
    m.set_plan(s, {"adjoint_warps": 0, "gap_forward": 0, "gap_backward": 0, "neighbour_sweep": sweep,
                   "pair_forward": 0})
    m.compute(s, desc=True)
    gi, gj, gs = m.pairs()
    oi, oj, os_ = oracle_pairs(batch, P.r_cut)
    assert len(gi) == len(oi)
    np.testing.assert_array_equal(gi, oi)
    np.testing.assert_array_equal(gj, oj)
    np.testing.assert_array_equal(gs, os_)
    assert len(gi) / 300 > 2.0 * 0.15 * 4.18879 * 125  # well above the mean-density estimate


# ------------------------------------------------------------------ GAP products: 1 or 3 FP16 terms
@pytest.mark.parametrize("name,m_sparse,expect", [("box100k_n10l10", None, 1),
                                                  ("twospecies4096_n8l8", 300, 3)])
def test_gap_terms_follow_the_probe_error(name, m_sparse, expect):
    """The number of FP16 products of the energy is chosen per model from the one-product
    error of the sparse rows' own energies: 4000 carbon-like rows lose ~3e-6 (one product);
    300 rows of the two-species box ~1e-4 (three products)."""
    P, qs, al, zeta = sparse_model(name, m_sparse)
    m = model_for(params_dict(P), "mixed", qs, al, zeta)
    terms, probe = m.gap_terms()
    print(f"PARITY {name} M={len(qs)}: one-product probe error {probe:.2e} -> {terms} products")
    assert terms == expect
    assert (probe <= 1e-5) == (expect == 1)


def test_gap_terms_forced_one_and_three_against_oracle():
    """Forced one and three products on the 64-atom box against the oracle's energies: three
    products leave only the descriptors' own error; the automatic choice equals one of them."""
    w = synth.get_workload("box64_n6l6")
    batch = w.structures()
    P, qs, al, zeta = sparse_model("box64_n6l6")
    ref = gap.evaluate(batch, P, qs, al, zeta, W=oracle_W(P.n_max, P.r_cut, P.sigma_r0), forces=False,
                       virial=False)
    m = model_for(params_dict(P), "mixed", qs, al, zeta)
    auto, probe = m.gap_terms()
    errs = {}
    for t in (1, 3):
        m.set_gap_terms(t)
        assert m.gap_terms()[0] == t
        e = m.compute(structures(batch), energy=True)["e_atom"].double().cpu().numpy()
        errs[t] = rel_all(e[None], ref["e_atom"][None])
    m.set_gap_terms(0)
    assert m.gap_terms()[0] == auto
    print(f"PARITY box64 forced products: one {errs[1]:.2e}, three {errs[3]:.2e} (probe {probe:.2e}, "
          f"automatic {auto})")
    assert errs[3] < 2e-6 and errs[1] < MIXED["e"]
    assert errs[3] < errs[1]


# ------------------------------------------------------------------ adjoint variants
@pytest.mark.parametrize("name,m_sparse,sampled", [("box64_n6l6", None, False), ("box1000_n8l8", 100, False),
                                                   ("twospecies4096_n8l8", 300, True),
                                                   ("box100k_n10l10", None, True)])
def test_adjoint_variants_against_oracle(name, m_sparse, sampled):
    """The adjoint on tcgen05 (TMEM accumulators) and on mma.sync with 2 and 4 warps per
    block, forced through the tile plan: forces against the oracle (all atoms, or 4 sampled
    atoms of the large boxes) within the mixed bar, and against each other."""
    w = synth.get_workload(name)
    batch = w.structures()
    P, qs, al, zeta = sparse_model(name, m_sparse)
    model = model_for(params_dict(P), "mixed", qs, al, zeta)
    s = structures(batch)
    model.compute(s, energy=True)
    W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
    if sampled:
        atoms = np.random.default_rng(7).choice(batch.n_atoms, 4, replace=False)
        f_ref, atoms = gap.forces_at(batch, P, qs, al, zeta, atoms, W=W)
    else:
        atoms = np.arange(batch.n_atoms)
        f_ref = gap.evaluate(batch, P, qs, al, zeta, W=W, virial=False)["forces"]
    forces = {}
    for variant in (5, 4, 2):
        model.set_plan(s, {"adjoint_warps": variant, "gap_forward": 0, "gap_backward": 0,
                           "neighbour_sweep": 0, "pair_forward": 0})
        f = model.compute(s, energy=True, forces=True)["forces"].cpu().numpy()
        forces[variant] = f
        err = rel_all(f[atoms], f_ref)
        print(f"PARITY {name} adjoint variant {variant}: F {err:.2e}")
        assert err < MIXED["f"]
    assert rel_all(forces[5], forces[4]) < 1e-5
    assert rel_all(forces[2], forces[4]) < 1e-5


def test_adjoint_variants_on_dense_cluster_and_empty_structures():
    """Edges of the tcgen05 adjoint and the per-bin neighbour sweep, forced through the tile
    plan: atoms squeezed into a corner (~470 pairs per atom: several 128-pair MMA tiles per
    atom, and bins over the shared-memory capacity), and a batch with empty structures and an
    isolated atom; forces against the oracle and against the mma.sync kernel."""
    P = Params(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, n_max=6, l_max=6)
    W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
    qs = soap.descriptors(synth.concat([synth.random_box(24, density=0.15, dmin=1.2, seed=43)]), P,
                          W=W)["q"].numpy()
    al = synth.gap_weights(len(qs), 44)
    base = synth.random_box(300, density=0.15, dmin=1.2, seed=41)
    dense = synth.concat([base])
    dense.pos[:] = dense.pos * 0.55
    lone = synth.Structure(pos=np.array([[5.0, 5.0, 5.0]]), cell=np.eye(3) * 20.0,
                           species=np.zeros(1, np.int32))
    empty = synth.Structure(pos=np.zeros((0, 3)), cell=np.eye(3) * 9.0, species=np.zeros(0, np.int32))
    ragged = synth.concat([empty, lone, synth.random_box(16, side=5.0, dmin=1.2, seed=3), empty])
    for batch, atoms in ((dense, np.array([0, 150])), (ragged, None)):
        model = model_for(params_dict(P), "mixed", qs, al, 2.0)
        s = structures(batch)
        model.compute(s, energy=True)
        if atoms is None:
            ref = gap.evaluate(batch, P, qs, al, 2.0, W=W, virial=False)
            f_ref, idx, e_ref = ref["forces"], np.arange(batch.n_atoms), ref["e_struct"]
        else:
            f_ref, idx = gap.forces_at(batch, P, qs, al, 2.0, atoms, W=W)
            e_ref = None
        got = {}
        for variant, sweep in ((5, 1), (4, 2)):
            model.set_plan(s, {"adjoint_warps": variant, "gap_forward": 0, "gap_backward": 0,
                               "neighbour_sweep": sweep, "pair_forward": sweep})
            out = model.compute(s, energy=True, forces=True)
            f = out["forces"].cpu().numpy()
            got[variant] = f
            err = rel_all(f[idx], f_ref)
            print(f"PARITY edges {batch.n_atoms} atoms, adjoint {variant}, sweep {sweep}: F {err:.2e}")
            assert err < MIXED["f"]
            if e_ref is not None:
                e = out["e_struct"].cpu().numpy()
                assert np.allclose(e, e_ref, rtol=MIXED["e"], atol=1e-12)
                assert e[0] == 0.0 and e[3] == 0.0 and np.all(f[0] == 0.0)
        assert rel_all(got[5], got[4]) < 1e-5


# ------------------------------------------------------------------ forward kernel variants
FORWARD_CASES = ["box64_n6l6", "box1000_n8l8", "twospecies4096_n8l8", "timing_n3l3", "timing_n12l12",
                 "timing_n11l12", "timing_n12l3", "timing_n10l10", "hp0", "hp1", "hp2", "hp3", "hp4",
                 "dense_cluster", "ragged"]


def forward_case(case, golden):
    """(params, batch, sampled centres or None for all atoms) of a forward-kernel case."""
    g66 = Params(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, n_max=6, l_max=6)
    if case.startswith("box") or case.startswith("twospecies"):
        w = synth.get_workload(case)
        b = w.structures()
        return Params.from_dict(w.params()), b, np.arange(0, b.n_atoms, max(1, b.n_atoms // 40))
    if case.startswith("timing"):
        n, l = (int(x) for x in case[len("timing_n"):].split("l"))
        P = Params(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, n_max=n, l_max=l)
        return P, TIMING_BOX, np.random.default_rng(n * 100 + l).choice(TIMING_BOX.n_atoms, 8, replace=False)
    if case.startswith("hp"):
        k = int(case[2:])
        return hp_variants(golden)[k], synth.concat([synth.random_box(40, side=7.5, dmin=1.0, seed=40 + k)]), None
    if case == "dense_cluster":
        dense = synth.concat([synth.random_box(300, density=0.15, dmin=1.2, seed=41)])
        dense.pos[:] = dense.pos * 0.55
        return g66, dense, np.array([0, 77, 150, 299])
    lone = synth.Structure(pos=np.array([[5.0, 5.0, 5.0]]), cell=np.eye(3) * 20.0,
                           species=np.zeros(1, np.int32))
    empty = synth.Structure(pos=np.zeros((0, 3)), cell=np.eye(3) * 9.0, species=np.zeros(0, np.int32))
    return g66, synth.concat([empty, lone, synth.random_box(16, side=5.0, dmin=1.2, seed=3), empty]), None


@pytest.mark.parametrize("case", FORWARD_CASES)
def test_forward_variants_against_oracle(case, golden):
    """Both forward pair kernels, forced through the tile plan (1 = FP32 FMA contraction,
    2 = tensor-core contraction with FP16 hi/lo operands), against the oracle's descriptors
    (sampled centres on the larger boxes) and against each other: basis sizes 3..12, the
    paper's hyperparameter sets, two species, a dense cluster (several 32-pair batches per
    atom) and a batch with empty structures and an isolated atom."""
    P, batch, centers = forward_case(case, golden)
    m = model_for(params_dict(P), "mixed")
    s = structures(batch)
    m.compute(s, desc=True)
    outs = {}
    for v in (1, 2):
        m.set_plan(s, {"adjoint_warps": 0, "gap_forward": 0, "gap_backward": 0, "neighbour_sweep": 0,
                       "pair_forward": v})
        out = m.compute(s, desc=True)
        outs[v] = out["q"].double().cpu().numpy() * out["pnorm"].double().cpu().numpy()[:, None]
        if centers is None:
            ref = soap.descriptors(batch, P, W=oracle_W(P.n_max, P.r_cut, P.sigma_r0))
            c = ref["centers"]
            err = rel_rows(outs[v][c], (ref["q"] * ref["pnorm"][:, None]).numpy())
        else:
            err = sampled_p_error(batch, P, out, centers)
        print(f"PARITY forward variant {v} {case}: p {err:.2e}")
        assert err < MIXED["p"]
    assert rel_rows(outs[2], outs[1]) < 1e-5


@pytest.mark.parametrize("n_max,l_max", [(12, 12), (8, 8)])
def test_tcgen05_adjoint_every_image_layout(n_max, l_max):
    """The tcgen05 adjoint reads its per-atom G operand from an image: two harmonic rows per
    128-byte row when the split rows take 64 bytes (n_max <= 10), one per row at n_max = 12;
    and a G buffer in shared memory when there are several species.  n = l = 12 (one species)
    and n = l = 8 with two species, forced through the tile plan, against the oracle's forces
    and the mma.sync kernel's."""
    nsp = 2 if n_max == 8 else 1
    P = Params(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, n_max=n_max, l_max=l_max, n_species=nsp)
    W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
    probs = [0.6, 0.4] if nsp == 2 else None
    batch = synth.concat([synth.random_box(48, density=0.12, dmin=1.1, seed=51, species_probs=probs)])
    sb = synth.concat([synth.random_box(20, density=0.12, dmin=1.1, seed=52, species_probs=probs)])
    qs = soap.descriptors(sb, P, W=W)["q"].numpy()
    al = synth.gap_weights(len(qs), 53)
    ref = gap.evaluate(batch, P, qs, al, 3.0, W=W, virial=False)["forces"]
    model = model_for(params_dict(P), "mixed", qs, al, 3.0)
    s = structures(batch)
    model.compute(s, energy=True)
    forces = {}
    for variant in (5, 4):
        model.set_plan(s, {"adjoint_warps": variant, "gap_forward": 0, "gap_backward": 0,
                           "neighbour_sweep": 0, "pair_forward": 0})
        forces[variant] = model.compute(s, energy=True, forces=True)["forces"].cpu().numpy()
        err = rel_all(forces[variant], ref)
        print(f"PARITY n={n_max} l={l_max} species {nsp}: adjoint variant {variant}: F {err:.2e}")
        assert err < MIXED["f"]
    assert rel_all(forces[5], forces[4]) < 1e-5
