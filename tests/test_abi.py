"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(tns_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_11424_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_five_hot_path_calls():
    names = _declared()
    for n in ("tns_build_lattice", "tns_apply_gate_layer", "tns_bp_gauge", "tns_sample", "tns_amplitude"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2507_11424_gb300 import _native
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _native.SIGNATURES, name


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2507_11424_gb300 import _native
    with pytest.raises(RuntimeError):
        _native.open_library(str(tmp_path / "missing.so"))


def test_error_string_available(lib):
    lib.tns_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.tns_last_error(), bytes)


def test_invalid_arguments_rejected_before_any_device_work(lib):
    """Host-side validation: NULL outputs / sizes are rejected with TNS_ERR_ARG without touching a GPU."""
    lib.tns_build_lattice.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.tns_build_lattice(0, None, 0, None, None, 4, 1, None, ctypes.byref(out)) == 1
    assert lib.tns_build_lattice(1, None, 0, None, None, 4, 1, None, None) == 1
    lib.tns_sample.restype = ctypes.c_int
    assert lib.tns_sample(None, 4, 1, ctypes.c_uint64(0), None, None, None) == 1


def test_learned_proposal_and_mh_reject_invalid_arguments(lib):
    """The MADE / MH entry points validate sizes and pointers on the host."""
    from paper_2507_11424_gb300 import _native
    L = _native.open_library(_native.LIB_PATH)
    out = ctypes.c_void_p()
    params = (ctypes.c_float * 8)()
    assert L.tns_made_create(1, 4, params, None, ctypes.byref(out)) == 1          # n_sites < 2
    assert L.tns_made_create(4, 0, params, None, ctypes.byref(out)) == 1          # hidden < 1
    assert L.tns_made_create(4, 4, None, None, ctypes.byref(out)) == 1            # no parameters
    assert L.tns_made_train(None, None, 1, 1, 1, None, 1e-3, None) == 1
    assert L.tns_made_grad(None, None, 1, None, None) == 1
    assert L.tns_made_logprob(None, None, 1, None) == 1
    assert L.tns_made_sample(None, 1, ctypes.c_uint64(0), None, None) == 1
    assert L.tns_made_params(None, None) == 1
    assert L.tns_mh_independent(-1, 4, None, None, None, None, ctypes.c_uint64(0), None, None, None) == 1
    assert L.tns_mh_independent(2, 3, None, None, None, None, ctypes.c_uint64(0), None, None, None) == 1
    assert L.tns_mh_independent(0, 3, None, None, None, None, ctypes.c_uint64(0), None, None, None) == 0


def test_contraction_test_entry_rejects_bad_mode(lib):
    from paper_2507_11424_gb300 import _native
    L = _native.open_library(_native.LIB_PATH)
    d = (ctypes.c_int64 * 1)(1)
    assert L.tns_test_contract(b"a", d, d, 0, None, b"a", d, d, 0, None, b"a", d, d, None, 0, None) == 1
    assert L.tns_test_contract(b"a", d, d, 0, d, b"a", d, d, 0, d, b"a", d, d, d, 7, None) == 1
