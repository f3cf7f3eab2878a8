"""The C-ABI library loads and exports every entry point include/qkc.h declares (CPU)."""
import ctypes
import re
from pathlib import Path

HEADER = Path(__file__).resolve().parents[1] / "include" / "qkc.h"


def declared():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qkc_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(native_lib):
    names = declared()
    assert {"qkc_compile", "qkc_load_ac", "qkc_set_params", "qkc_evaluate", "qkc_marginals", "qkc_gradient",
            "qkc_sample"} <= set(names)
    for n in names:
        assert hasattr(native_lib, n), n


def test_last_error_after_bad_call(native_lib):
    from paper_2103_17226_gb300 import native as N
    out = ctypes.c_void_p()
    n = ctypes.c_uint64()
    st = native_lib.qkc_compile(None, 0, 0, 0, 1, 0, 0, ctypes.byref(out), ctypes.byref(n))
    assert st == 1
    assert b"qkc_compile" in native_lib.qkc_last_error()


def test_library_has_sm103a_kernels():
    from paper_2103_17226_gb300.build import build_library
    lib = build_library()
    data = lib.read_bytes()
    assert b"sm_103a" in data or b"sm_103" in data
