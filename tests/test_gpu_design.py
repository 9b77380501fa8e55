"""Parity of the sparse-GAP fitting matrices (soapgap_design, soapgap_kernel_rows) with the
FP64 oracle (oracle.gap.kernel_matrix, structure_rows, kernel_gradients).

Bars (a kernel row entry is the energy of a one-environment model with unit weight, so
the rows take the energy bar of the evaluation; the mixed descriptors carry p errors up to
1e-5, and k = S^zeta amplifies |dq| <= 2e-5 by zeta):
  kernel rows       mixed: max |dk| <= 1e-4 (k in [0, 1]); FP64: 1e-10
  energy rows       relative per entry 1e-4 (mixed), 1e-10 (FP64)
  force rows        mixed: |d dk|_2 / |dk|_2 <= 1e-3 over the whole matrix (the forces bar;
                    single FP16 products of centred, scaled operands give ~1e-4);
                    FP64: 1e-9
At the full size of the 256-structure training batch: sampled atoms and sparse columns
against the oracle, the force identity F = -dk alpha against the evaluation path, and a
zero sum over every structure (translation invariance).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import Params, gap, soap

from parity_helpers import oracle_W, rel_all, sparse_model

pytestmark = pytest.mark.gpu

TOL = {"mixed": dict(k=1e-4, ks=1e-4, dk=1e-3), "fp64": dict(k=1e-10, ks=1e-10, dk=1e-9)}


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_02142_gb300 import build
    build.build()


def params_dict(P: Params):
    return dict(r_cut=P.r_cut, r_soft=P.r_soft, sigma_r0=P.sigma_r0, sigma_p0=P.sigma_p0,
                alpha_r=P.alpha_r, alpha_p=P.alpha_p, amp_a=P.amp_a, n_f=P.n_f,
                central_weight=P.central_weight, n_max=P.n_max, l_max=P.l_max,
                n_species=P.n_species, eq08_weight=P.eq08_weight)


def make(name, m, precision):
    from paper_1905_02142_gb300.api import SoapGap
    P, qs, al, zeta = sparse_model(name, m)
    model = SoapGap.from_dict(params_dict(P), precision=precision)
    model.set_model(qs, al, zeta)
    return model, P, qs, al, zeta


def structures(batch):
    from paper_1905_02142_gb300.api import Structures
    return Structures.from_batch(batch)


CASES = {
    # 64-atom box of the descriptor workload, its 32 sparse environments
    "box64": lambda: (synth.get_workload("box64_n6l6").structures(), "box64_n6l6", 32),
    # ten ragged structures (4..150 atoms) with the training-batch hyperparameters
    "batch": lambda: (synth.batched_boxes(10, n_lo=4, n_hi=150, seed=77), "batch256_n8l8", 24),
    # two species: channel blocks of the Jacobian
    "two_species": lambda: (synth.concat([synth.random_box(40, density=0.10, dmin=1.0, seed=41,
                                                           species_probs=(0.7, 0.3))]),
                            "twospecies4096_n8l8", 16),
    # 7 atoms in a sheared 3.1 A cell with r_cut 5: many self-images (pairs i -> i + S)
    "self_images": lambda: (synth.concat([synth.random_box(7, side=3.1, dmin=1.0, seed=5,
                                                           shear=0.35)]), "box64_n6l6", 12),
}


@pytest.fixture(scope="module")
def oracle_rows():
    cache = {}

    def get(case):
        if case not in cache:
            batch, name, m = CASES[case]()
            P, qs, al, zeta = sparse_model(name, m)
            W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
            q = soap.descriptors(batch, P, W=W)["q"]
            k = gap.kernel_matrix(q, qs, zeta)
            cache[case] = dict(batch=batch, name=name, m=m, k=k.numpy(),
                               ks=gap.structure_rows(k, batch.atom_offs).numpy(),
                               dk=gap.kernel_gradients(batch, P, qs, zeta, W=W))
        return cache[case]
    return get


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("case", list(CASES))
def test_design_rows_match_oracle(case, precision, oracle_rows):
    ref = oracle_rows(case)
    model, P, qs, al, zeta = make(ref["name"], ref["m"], precision)
    out = model.design(structures(ref["batch"]), k_atom=True, k_struct=True, dk=True)
    k = out["k_atom"].double().cpu().numpy()
    ks = out["k_struct"].cpu().numpy()
    dk = out["dk"].double().cpu().numpy()
    tol = TOL[precision]
    err_k = np.abs(k - ref["k"]).max()
    err_ks = np.max(np.abs(ks - ref["ks"]) / np.abs(ref["ks"]))
    err_dk = rel_all(dk, ref["dk"])
    print(f"{case} {precision}: k {err_k:.2e}  k_struct {err_ks:.2e}  dk {err_dk:.2e}")
    assert err_k < tol["k"]
    assert err_ks < tol["ks"]
    assert err_dk < tol["dk"]
    # every atom's rows: no target left out or written twice
    norms = np.linalg.norm(ref["dk"], axis=(1, 2))
    per_atom = np.linalg.norm(dk - ref["dk"], axis=(1, 2)) / np.maximum(norms, 1e-3 * norms.max())
    assert per_atom.max() < 20 * tol["dk"]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_design_edge_cases(precision):
    """An empty structure, an isolated atom (no neighbour, no image within r_cut) and a
    small box in one batch, with a non-integer zeta (the clamped power of Sec. I)."""
    from paper_1905_02142_gb300.api import SoapGap
    batch = synth.concat([synth.random_box(0, side=9.0, seed=1), synth.random_box(1, side=20.0, seed=2),
                          synth.random_box(12, side=5.0, dmin=1.2, seed=3)])
    w = synth.get_workload("box64_n6l6")
    P = Params.from_dict(w.params())
    W = oracle_W(P.n_max, P.r_cut, P.sigma_r0)
    P_, qs, al, _ = sparse_model("box64_n6l6", 8)
    zeta = 2.5
    model = SoapGap.from_dict(params_dict(P), precision=precision)
    model.set_model(qs, al, zeta)
    out = model.design(structures(batch), k_atom=True, k_struct=True, dk=True)
    q = soap.descriptors(batch, P, W=W)["q"]
    k_ref = gap.kernel_matrix(q, qs, zeta).numpy()
    ks_ref = gap.structure_rows(k_ref, batch.atom_offs).numpy()
    dk_ref = gap.kernel_gradients(batch, P, qs, zeta, W=W)
    k = out["k_atom"].double().cpu().numpy()
    ks = out["k_struct"].cpu().numpy()
    dk = out["dk"].double().cpu().numpy()
    tol = TOL[precision]
    assert np.all(ks[0] == 0.0)                      # the empty structure
    assert np.all(dk[0] == 0.0)                      # the isolated atom does not move anything
    assert np.abs(k - k_ref).max() < tol["k"]
    assert np.max(np.abs(ks[1:] - ks_ref[1:]) / np.abs(ks_ref[1:])) < tol["ks"]
    assert rel_all(dk, dk_ref) < tol["dk"]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_sparse_block(precision):
    model, P, qs, al, zeta = make("box64_n6l6", 32, precision)
    kmm = model.kernel_rows(torch.as_tensor(qs, device="cuda")).double().cpu().numpy()
    ref = gap.kernel_matrix(qs, qs, zeta).numpy()
    assert np.abs(kmm - ref).max() < TOL[precision]["k"]
    assert np.abs(np.diag(kmm) - 1.0).max() < TOL[precision]["k"]


def test_selected_outputs_only():
    batch, name, m = CASES["batch"]()
    model, P, qs, al, zeta = make(name, m, "mixed")
    s = structures(batch)
    full = model.design(s, k_atom=True, k_struct=True, dk=True)
    only_ks = model.design(s, k_struct=True)
    only_dk = model.design(s, dk=True)
    assert set(only_ks) == {"k_struct"} and set(only_dk) == {"dk"}
    assert torch.equal(only_ks["k_struct"], full["k_struct"])
    assert rel_all(only_dk["dk"].cpu().numpy(), full["dk"].cpu().numpy()) < 1e-6


def test_design_needs_model_and_valid_flags():
    import ctypes
    from paper_1905_02142_gb300 import _lib as L
    from paper_1905_02142_gb300.api import SoapGap
    w = synth.get_workload("box64_n6l6")
    b = structures(w.structures()).c_batch()
    bare = SoapGap.from_dict(w.params(), precision="mixed")
    assert bare.lib.soapgap_design(bare.h, ctypes.byref(b), 0, None, None, None, None) == L.E_STATE
    model, *_ = make("box64_n6l6", 8, "mixed")
    assert model.lib.soapgap_design(model.h, ctypes.byref(b), L.DESIGN_K, None, None, None,
                                    None) == L.E_INVALID_ARG          # DESIGN_K without k_atom
    assert model.lib.soapgap_design(model.h, ctypes.byref(b), 1 << 20, None, None, None,
                                    None) == L.E_INVALID_ARG          # unknown flag bit


def test_design_with_a_verlet_skin():
    """With a skin the list holds pairs up to r_cut + skin; pairs beyond r_cut give zero
    columns, so the rows equal those of a list without skin (up to summation order)."""
    batch, name, m = CASES["batch"]()
    model, *_ = make(name, m, "mixed")
    s = structures(batch)
    plain = model.design(s, k_atom=True, k_struct=True, dk=True)
    model.set_skin(0.6)
    skinned = model.design(s, k_atom=True, k_struct=True, dk=True)
    assert model.pair_count() > 0
    assert torch.allclose(skinned["k_atom"], plain["k_atom"], rtol=0, atol=1e-6)
    assert torch.allclose(skinned["k_struct"], plain["k_struct"], rtol=1e-6, atol=0)
    assert rel_all(skinned["dk"].cpu().numpy(), plain["dk"].cpu().numpy()) < 1e-5


# ------------------------------------------------------------------ full training batch
@pytest.fixture(scope="module")
def full_batch():
    w = synth.get_workload("batch256_n8l8")
    batch = w.structures()
    model, P, qs, al, zeta = make("batch256_n8l8", None, "mixed")
    s = structures(batch)
    out = model.design(s, k_struct=True, dk=True)
    return w, batch, model, P, qs, al, zeta, s, out


def test_full_batch_force_identity_and_translation(full_batch):
    w, batch, model, P, qs, al, zeta, s, out = full_batch
    dk = out["dk"].double()
    al_t = torch.as_tensor(al, device="cuda")
    f_rows = -(dk @ al_t)                                        # [N, 3]
    ev = model.compute(s, energy=True, forces=True)
    assert rel_all(f_rows.cpu().numpy(), ev["forces"].cpu().numpy()) < 2e-3
    e_rows = out["k_struct"] @ al_t
    assert np.max(np.abs((e_rows - ev["e_struct"]).cpu().numpy()) /
                  np.abs(ev["e_struct"].cpu().numpy())) < 1e-4
    offs = batch.atom_offs
    sums = torch.stack([dk[offs[t]:offs[t + 1]].sum(dim=0) for t in range(batch.n_struct)])
    assert float(sums.norm() / dk.norm()) < 1e-3


def test_full_batch_sampled_against_oracle(full_batch):
    w, batch, model, P, qs, al, zeta, s, out = full_batch
    rng = np.random.default_rng(11)
    atoms = np.sort(rng.choice(batch.n_atoms, 3, replace=False))
    sparse = np.sort(rng.choice(len(qs), 4, replace=False))
    ref = gap.kernel_gradients(batch, P, qs, zeta, atoms=atoms, sparse=sparse,
                               W=oracle_W(P.n_max, P.r_cut, P.sigma_r0))
    got = out["dk"][torch.as_tensor(atoms)][:, :, torch.as_tensor(sparse)].double().cpu().numpy()
    assert rel_all(got, ref) < TOL["mixed"]["dk"]
