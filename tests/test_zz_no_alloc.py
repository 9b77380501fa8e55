"""The allocation-free GAP energy entry point (soapgap_gap_energy_noalloc), called through
the C ABI, against the regular entry point (soapgap_compute) on the same inputs.

It serves callers that cannot allocate device memory (their own memory pool, or no
tolerance for the synchronisation an allocation may cause); its scratch sits in a fixed
device array inside the library.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

from parity_helpers import sparse_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_02142_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_noalloc_energies_match_regular_entry_point_twice(lib):
    from paper_1905_02142_gb300 import _lib as L
    from paper_1905_02142_gb300.api import SoapGap, Structures
    P, qs, al, zeta = sparse_model("box64_n6l6")
    model = SoapGap.from_dict(dict(r_cut=P.r_cut, r_soft=P.r_soft, sigma_r0=P.sigma_r0,
                                   sigma_p0=P.sigma_p0, n_max=P.n_max, l_max=P.l_max),
                              precision="mixed")
    model.set_model(qs, al, zeta)
    qs_d = torch.as_tensor(qs, dtype=torch.float32, device="cuda").contiguous()
    al_d = torch.as_tensor(al, dtype=torch.float32, device="cuda").contiguous()
    st = torch.cuda.current_stream().cuda_stream
    # descriptors and regular energies of two boxes first, so that no torch or handle
    # allocation falls between the two allocation-free calls below
    cases = []
    for seed, n_atoms in ((61, 48), (62, 20)):   # two calls in a row, different sizes
        batch = synth.concat([synth.random_box(n_atoms, side=7.0, dmin=1.2, seed=seed)])
        out = model.compute(Structures.from_batch(batch), desc=True, energy=True)
        e = torch.full((n_atoms,), float("nan"), dtype=torch.float32, device="cuda")
        cases.append((n_atoms, out["q"], out["e_atom"].double().cpu().numpy(), e))
    torch.cuda.synchronize()
    free = []
    for n_atoms, q, ref, e in cases:
        rc = lib.soapgap_gap_energy_noalloc(q.data_ptr(), qs_d.data_ptr(), al_d.data_ptr(),
                                            n_atoms, len(qs), model.dim, zeta, e.data_ptr(), st)
        assert rc == L.OK
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got = e.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4
    # the first call may load the library's module; the second one must leave the
    # device's free memory exactly as it was
    assert free[1] == free[0]


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_1905_02142_gb300 import _lib as L
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    p = dummy.data_ptr()
    # 4194304 floats of scratch: 65537 atoms x 64 tiles (m = 4096) is one row too many
    rc = lib.soapgap_gap_energy_noalloc(p, p, p, 65537, 4096, 8, 2.0, p, None)
    assert rc == L.E_CAPACITY
    # one sparse tile (m <= 64) keeps the scratch small, but 4194304 atoms need 65536
    # block rows of 64, one more than a launch grid holds
    rc = lib.soapgap_gap_energy_noalloc(p, p, p, 4194304, 64, 8, 2.0, p, None)
    assert rc == L.E_CAPACITY
    rc = lib.soapgap_gap_energy_noalloc(p, p, p, 4, 0, 8, 2.0, p, None)
    assert rc == L.E_INVALID_ARG
