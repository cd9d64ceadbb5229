"""The C-ABI library loads and exports every entry point include/spmv.h declares
(no compute calls: this runs without a GPU), and host-side argument checks
answer before any CUDA work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spmv.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1805_11938_gb300 import build

    build.build()
    import paper_1805_11938_gb300 as sp

    return sp.lib()


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^SPMV_API [^;(]*?\b(spmv_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = declared()
    for n in ("spmv_convert", "spmv_run", "spmv_to_csr", "spmv_features", "spmv_select", "spmv_free",
              "spmv_batch_build", "spmv_batch_run", "spmv_strerror"):
        assert n in names


def test_every_declared_symbol_exported(lib):
    from paper_1805_11938_gb300 import _abi

    for n in declared():
        assert hasattr(lib, n), n
    assert set(declared()) == set(_abi.EXPORTED)


def test_host_side_argument_errors(lib):
    import paper_1805_11938_gb300 as sp

    assert lib.spmv_version() >= 100
    assert lib.spmv_strerror(-3) == b"footprint above the cap"
    out = ctypes.c_void_p()
    # NULL csr, bad format and empty shapes are rejected before any CUDA call
    assert lib.spmv_convert(0, None, None, None, ctypes.byref(out)) == -1
    c = sp._abi.spmv_csr(0, 5, 0, None, None, None)
    assert lib.spmv_convert(0, ctypes.byref(c), None, None, ctypes.byref(out)) == -1
    assert lib.spmv_convert(9, ctypes.byref(c), None, None, ctypes.byref(out)) == -1
    assert b"unknown format" in lib.spmv_last_error()
    assert lib.spmv_run(None, None, None, None) == -1
    assert lib.spmv_select(None, None, None, None) == -5
    assert lib.spmv_batch_build(None, 0, None, None) == -1
