"""ctypes binding of the C ABI declared in include/tns.h and include/tns_testing.h.

Argument marshalling only.

Every step of the method runs inside libtns.so; this module converts Python and
torch arguments into plain pointers and sizes.  Loading fails loudly when the
library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtns.so")

TNS_OK, TNS_ERR_ARG, TNS_ERR_CUDA, TNS_ERR_OOM, TNS_ERR_NOT_CONVERGED, TNS_ERR_NUMERIC, TNS_ERR_STATE = range(7)
PREC = {"fp64": 0, "mixed": 1}
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_CUDA", "ERR_OOM", "ERR_NOT_CONVERGED", "ERR_NUMERIC", "ERR_STATE"]

# name -> (restype, argtypes), mirroring include/tns.h
SIGNATURES = {
    "tns_build_lattice": (C.c_int, [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int,
                                    C.c_void_p, C.POINTER(C.c_void_p)]),
    "tns_apply_gate_layer": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_double,
                                       C.c_void_p]),
    "tns_bp_gauge": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "tns_sample": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_sample_range": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "tns_sample_replay": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "tns_amplitude": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_log_fidelity": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "tns_bp_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "tns_log_norm": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double)]),
    "tns_set_precision": (C.c_int, [C.c_void_p, C.c_int]),
    "tns_set_tensor_cores": (C.c_int, [C.c_void_p, C.c_int32]),
    "tns_set_compression": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "tns_set_graphs": (C.c_int, [C.c_void_p, C.c_int32]),
    "tns_certify": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_test_tc_tile": (C.c_int, [C.c_int32]),
    "tns_direct_marginals": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "tns_query": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                            C.POINTER(C.c_int32)]),
    "tns_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "tns_load": (C.c_int, [C.c_char_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "tns_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "tns_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "tns_profile_read": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double)]),
    "tns_eigh_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_eigh_noalloc_status": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p]),
    "tns_test_env_site": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_made_create": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "tns_made_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tns_made_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_float,
                                 C.c_void_p]),
    "tns_made_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_double)]),
    "tns_made_logprob": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "tns_made_sample": (C.c_int, [C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p]),
    "tns_made_destroy": (None, [C.c_void_p]),
    "tns_mh_independent": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_destroy": (None, [C.c_void_p]),
    "tns_test_philox": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_test_eigh": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_test_eigh32": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_test_eigh_sweeps": (C.c_int, [C.c_int32, C.c_void_p]),
    "tns_test_cholw": (C.c_int, [C.c_int32, C.c_int32, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_test_tcgemm": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_test_contract": (C.c_int, [C.c_char_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_char_p, C.c_void_p,
                                    C.c_void_p, C.c_int32, C.c_void_p, C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int32, C.c_void_p]),
    "tns_test_plan": (C.c_int, [C.c_char_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_char_p, C.c_void_p, C.c_void_p,
                                C.c_int32, C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tns_test_svd": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    "tns_last_error": (C.c_char_p, []),
}

_lib = None


def open_library(path: str):
    """dlopen a libtns.so and declare the C signatures; raises if the file is missing."""
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: str = LIB_PATH):
    """The process-wide libtns.so handle (loaded on first use)."""
    global _lib
    if _lib is None:
        _lib = open_library(path)
    return _lib


class TNSError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        self.code = code
        name = STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else str(code)
        super().__init__(f"{where}: TNS_{name}: {msg}")


def check(code: int, where: str, allow=()):
    if code != TNS_OK and code not in allow:
        raise TNSError(code, where, (load().tns_last_error() or b"").decode(errors="replace"))
    return code
