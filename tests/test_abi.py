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
