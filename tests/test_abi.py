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


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field offset of the header's structs, compiled by the
    host C compiler, equal the ctypes structures the binding passes."""
    import shutil
    import subprocess

    from paper_1805_11938_gb300 import _abi

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda_inc = None
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime_api.h")):
            cuda_inc = os.path.join(d, "include")
    if cuda_inc is None:
        pytest.skip("CUDA headers not found")
    structs = {"spmv_csr": _abi.spmv_csr, "spmv_params": _abi.spmv_params, "spmv_info": _abi.spmv_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "spmv.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[f"{name} size"]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_probe_is_a_separate_library(lib):
    """The benchmark's gather probe is not part of the library's ABI: it lives in
    a shared library of its own, which exports exactly its two calls."""
    import subprocess

    from paper_1805_11938_gb300 import _abi, build, probe

    assert not hasattr(lib, "spmv_probe_gather")
    out = subprocess.run(["nm", "-D", "--defined-only", build.PROBE_LIB], capture_output=True, text=True).stdout
    syms = sorted(l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("spmv_"))
    assert syms == ["spmv_probe_gather", "spmv_probe_partials"]
    assert not any(n.startswith("spmv_probe") for n in _abi.EXPORTED)
    assert probe.LIB_PATH == build.PROBE_LIB
