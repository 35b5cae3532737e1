"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/csc.h declares (no compute calls here)."""
import ctypes
import shutil

import pytest

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not __import__("os").path.exists(
    "/usr/local/cuda/bin/nvcc"), reason="CUDA toolkit not available")


@pytest.fixture(scope="module")
def built():
    from paper_1602_02018_gb300 import build

    return build.build()


def test_every_header_symbol_is_exported(built):
    import paper_1602_02018_gb300 as csc

    L = ctypes.CDLL(built)
    names = csc.header_symbols()
    assert len(names) >= 18
    for name in names:
        assert hasattr(L, name), f"{name} declared in include/csc.h but not exported"


def test_binding_declares_every_symbol(built):
    from paper_1602_02018_gb300 import _native

    assert set(_native.header_symbols()) <= set(_native._SIGNATURES)


def test_status_strings_and_version(built):
    from paper_1602_02018_gb300 import _native

    L = _native.lib()
    assert L.csc_status_str(0) == b"CSC_OK"
    assert L.csc_status_str(5) == b"CSC_E_NOT_CONVERGED"
    assert b"sm_103a" in L.csc_version()


def test_header_constants_match_binding():
    """Every status code and flag #define of include/csc.h has the same value in the binding."""
    import os
    import re

    from paper_1602_02018_gb300 import _native

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "csc.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(CSC_[A-Z0-9_]+)\s+(\d+)u?\b", hdr)}
    for name in ("CSC_E_NUMERIC", "CSC_CHECK_FINITE", "CSC_CLENSHAW", "CSC_HIGHPASS", "CSC_VARDENSITY",
                 "CSC_E_UNSUPPORTED", "CSC_E_NOT_CONVERGED"):
        assert name in defs, name
    for name, value in defs.items():
        if hasattr(_native, name):
            assert getattr(_native, name) == value, name
