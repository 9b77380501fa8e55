"""The C-ABI library builds, loads, exports every declared symbol, and rejects bad
parameters on the host before any device work (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "soapgap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(soapgap_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1905_02142_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_constants():
    """Integer #defines of the header (SOAPGAP_X -> value), comments removed."""
    src = open(os.path.join(ROOT, "include", "soapgap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, val in re.findall(r"#define\s+SOAPGAP_([A-Z0-9_]+)\s+\(?(-?\d+)u?\)?", src):
        out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    """Every constant the Python binding mirrors (status codes, precisions, call flags, stage
    and plan lengths, peak kinds) has the header's value, and the name tuples have the
    header's lengths."""
    from paper_1905_02142_gb300 import _lib
    from paper_1905_02142_gb300.api import SoapGap
    hdr = declared_constants()
    mirrored = ["OK", "E_INVALID_ARG", "E_UNSUPPORTED", "E_CAPACITY", "E_CUDA", "E_STATE",
                "FP64", "MIXED", "DESC", "ENERGY", "FORCES", "VIRIAL", "TIMING", "ASYNC",
                "DESIGN_K", "DESIGN_KSTRUCT", "DESIGN_DK", "N_DESIGN_STAGES", "N_STAGES",
                "PLAN_LEN", "PEAK_FP32_FMA", "PEAK_FP64_FMA"]
    for name in mirrored:
        assert name in hdr, name
        assert getattr(_lib, name) == hdr[name], (name, getattr(_lib, name), hdr[name])
    assert len(_lib.STAGES) == hdr["N_STAGES"]
    assert len(_lib.DESIGN_STAGES) == hdr["N_DESIGN_STAGES"]
    assert len(SoapGap.PLAN_KEYS) == hdr["PLAN_LEN"]
    flags = [hdr[f] for f in ("DESC", "ENERGY", "FORCES", "VIRIAL", "TIMING", "ASYNC",
                              "DESIGN_K", "DESIGN_KSTRUCT", "DESIGN_DK")]
    assert all(f & (f - 1) == 0 for f in flags) and len(set(flags)) == len(flags)
    # the kernels size their per-species arrays by the library's own limit, which the
    # parameter check takes from the header
    common = open(os.path.join(ROOT, "paper_1905_02142_gb300", "csrc", "common.cuh")).read()
    assert int(re.search(r"#define\s+SG_MAX_SPECIES\s+(\d+)", common).group(1)) == hdr["MAX_SPECIES"]


def test_every_declared_symbol_is_exported(lib):
    from paper_1905_02142_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as strict C99 (no C++ in the ABI), and a C program can
    take the address of every declared function."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import subprocess
    names = declared_functions()
    src = tmp_path / "use_header.c"
    src.write_text('#include "soapgap.h"\n'
                   "void* table[] = {\n" + ",\n".join(f"  (void*){n}" for n in names) + "\n};\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-Wno-pedantic", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                        "-o", str(tmp_path / "use_header.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-x", "c", os.path.join(ROOT, "include", "soapgap.h")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_parameter_validation_happens_on_host(lib):
    from paper_1905_02142_gb300 import _lib as L

    def create(**over):
        base = dict(r_cut=5.0, r_soft=4.5, sigma_r0=0.5, sigma_p0=0.5, alpha_r=0.0, alpha_p=0.0,
                    amp_a=1.0, n_f=4.0, central_weight=1.0, n_max=8, l_max=8, n_species=1,
                    precision=L.MIXED, eq08_weight=0)
        base.update(over)
        p = L.Params(*[base[f] for f, _ in L.Params._fields_])
        h = ctypes.c_void_p()
        return lib.soapgap_create(ctypes.byref(p), ctypes.byref(h)), h

    for over, code in [({"n_max": 13}, L.E_UNSUPPORTED), ({"n_max": 1}, L.E_UNSUPPORTED),
                       ({"l_max": 13}, L.E_UNSUPPORTED), ({"n_species": 9}, L.E_UNSUPPORTED),
                       ({"r_soft": 6.0}, L.E_INVALID_ARG), ({"r_cut": -1.0}, L.E_INVALID_ARG),
                       ({"sigma_r0": 0.0}, L.E_INVALID_ARG), ({"alpha_r": -0.1}, L.E_INVALID_ARG),
                       ({"precision": 7}, L.E_INVALID_ARG), ({"eq08_weight": 2}, L.E_INVALID_ARG)]:
        rc, h = create(**over)
        assert rc == code, over
        assert not h.value


def test_null_handle_is_rejected(lib):
    from paper_1905_02142_gb300 import _lib as L
    d = ctypes.c_int32()
    assert lib.soapgap_descriptor_dim(None, ctypes.byref(d)) == L.E_INVALID_ARG
    assert lib.soapgap_compute(None, None, 0, None, None, None, None, None, None, None) == L.E_INVALID_ARG
    assert lib.soapgap_design(None, None, 0, None, None, None, None) == L.E_INVALID_ARG
    assert lib.soapgap_kernel_rows(None, None, 0, None, None) == L.E_INVALID_ARG
    assert lib.soapgap_design_times(None, None) == L.E_INVALID_ARG
    lib.soapgap_destroy(None)


@pytest.mark.parametrize("n_max,r_cut,sigma", [(2, 4.0, 0.5), (6, 3.7, 0.5), (8, 5.0, 0.5),
                                               (8, 4.3, 0.12), (10, 5.0, 0.5), (12, 4.5, 0.3)])
def test_library_orthonormaliser_matches_oracle(lib, n_max, r_cut, sigma):
    # both sides build W = S^-1/2 in extended precision (binary128 vs 40-digit mpmath) from
    # independent evaluations of S, then round to FP64: they must agree to a few ulps
    import numpy as np

    from oracle import basis
    w = np.zeros((n_max, n_max))
    assert lib.soapgap_orthonormaliser(n_max, r_cut, sigma, w.ctypes.data) == 0
    ref = basis.orthonormaliser(n_max, r_cut, sigma)
    assert np.abs(w - ref).max() <= 8 * np.finfo(float).eps * np.abs(ref).max()
    assert np.allclose(w, w.T, rtol=0, atol=4 * np.finfo(float).eps * np.abs(ref).max())
