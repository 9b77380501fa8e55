"""ctypes declarations of the C ABI in include/soapgap.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsoapgap.so")

OK = 0
E_INVALID_ARG = -1
E_UNSUPPORTED = -2
E_CAPACITY = -3
E_CUDA = -4
E_STATE = -5

FP64 = 0
MIXED = 1

DESC = 1
ENERGY = 2
FORCES = 4
VIRIAL = 8
TIMING = 16
ASYNC = 32
DESIGN_K = 64
DESIGN_KSTRUCT = 128
DESIGN_DK = 256
N_DESIGN_STAGES = 4
DESIGN_STAGES = ("descriptors", "kernel_rows", "jacobian", "force_rows")
N_STAGES = 7
PLAN_LEN = 5
PEAK_FP32_FMA = 0
PEAK_FP64_FMA = 1
STAGES = ("neighbours", "pair_forward", "power_spectrum", "gap_forward", "gap_backward",
          "pair_adjoint", "finish")

# every entry point the header declares: (name, restype, argtypes)
c_void_p, c_int32, c_int64, c_double, c_uint32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                                  ctypes.c_double, ctypes.c_uint32)


class Params(ctypes.Structure):
    _fields_ = [("r_cut", c_double), ("r_soft", c_double), ("sigma_r0", c_double),
                ("sigma_p0", c_double), ("alpha_r", c_double), ("alpha_p", c_double),
                ("amp_a", c_double), ("n_f", c_double), ("central_weight", c_double),
                ("n_max", c_int32), ("l_max", c_int32), ("n_species", c_int32),
                ("precision", c_int32), ("eq08_weight", c_int32)]


class Batch(ctypes.Structure):
    _fields_ = [("n_struct", c_int32), ("n_atoms", c_int32), ("atom_offs_host", c_void_p),
                ("cell_host", c_void_p), ("pos", c_void_p), ("species", c_void_p)]


SIGNATURES = {
    "soapgap_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(c_void_p)]),
    "soapgap_orthonormaliser": (ctypes.c_int, [c_int32, c_double, c_double, c_void_p]),
    "soapgap_descriptor_dim": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int32)]),
    "soapgap_set_model": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_double]),
    "soapgap_compute": (ctypes.c_int, [c_void_p, ctypes.POINTER(Batch), c_uint32, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "soapgap_backward": (ctypes.c_int, [c_void_p, ctypes.POINTER(Batch), c_void_p, c_void_p,
                                        c_void_p, c_void_p]),
    "soapgap_compute_host": (ctypes.c_int, [c_void_p, ctypes.POINTER(Batch), c_uint32, c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p]),
    "soapgap_tc_gemm_f16": (ctypes.c_int, [c_void_p, c_void_p, c_int32, c_void_p, c_int32, c_int32,
                                           c_void_p, c_void_p]),
    "soapgap_stage_times": (ctypes.c_int, [c_void_p, c_void_p]),
    "soapgap_last_launch_count": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int64)]),
    "soapgap_last_pair_count": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int64)]),
    "soapgap_export_pairs": (ctypes.c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "soapgap_gap_energy_noalloc": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                                  c_int32, c_double, c_void_p, c_void_p]),
    "soapgap_set_gap_terms": (ctypes.c_int, [c_void_p, c_int32]),
    "soapgap_gap_terms": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_double)]),
    "soapgap_measure_alu_peak": (ctypes.c_int, [c_int32, ctypes.POINTER(c_double),
                                                ctypes.POINTER(c_int32), c_void_p]),
    "soapgap_sync_status": (ctypes.c_int, [c_void_p, c_void_p]),
    "soapgap_autotune": (ctypes.c_int, [c_void_p, ctypes.POINTER(Batch), c_void_p, c_void_p]),
    "soapgap_get_plan": (ctypes.c_int, [c_void_p, ctypes.POINTER(Batch), c_void_p]),
    "soapgap_set_plan": (ctypes.c_int, [c_void_p, ctypes.POINTER(Batch), c_void_p]),
    "soapgap_set_skin": (ctypes.c_int, [c_void_p, c_double]),
    "soapgap_last_rebuild": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int32)]),
    "soapgap_verlet": (ctypes.c_int, [c_void_p, ctypes.POINTER(Batch), c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_double, c_int32, c_void_p]),
    "soapgap_design": (ctypes.c_int, [c_void_p, ctypes.POINTER(Batch), c_uint32, c_void_p, c_void_p,
                                      c_void_p, c_void_p]),
    "soapgap_design_times": (ctypes.c_int, [c_void_p, c_void_p]),
    "soapgap_kernel_rows": (ctypes.c_int, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "soapgap_last_error": (ctypes.c_char_p, [c_void_p]),
    "soapgap_destroy": (None, [c_void_p]),
}

_lib = None


def load():
    """Load the in-tree CUDA library; fail loudly if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1905_02142_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
