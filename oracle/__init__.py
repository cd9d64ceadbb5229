"""CPU ORACLE -- test infrastructure only.

Plain, slow, obviously correct reference for everything the library computes.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA path
(``paper_1805_11938_gb300``) and neither imports the other; the seeded input
generators in ``synth`` are the only common dependency.

* ``spmv_oracle.c`` (built with ``gcc -O2 -ffp-contract=off``): CSR SpMV
  (Sec. II-A), dense matvec, COO->CSR, and every layout of Sec. II-B / Table I
  (ELL, SELL-C-sigma, HYB, CSR5) with its way back to CSR.
* ``features`` / ``mlp`` (numpy, float64): the 16 matrix features (Table IV
  plus eight defined here), their scaling (Sec. V-B "Feature Scaling"), and
  the selector network's forward pass, cross-entropy gradient and Adam step.

Every function is pinned by ``tests/test_oracle_pins.py`` against something
other than itself (Table I, closed forms, exact integer arithmetic, dense
library matvec, brute force, finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .features import FEATURE_NAMES, features, hyb_k_of_lengths  # noqa: F401
from . import mlp  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_F64P = ctypes.POINTER(ctypes.c_double)
_U8P = ctypes.POINTER(ctypes.c_uint8)
_I32, _I64 = ctypes.c_int32, ctypes.c_int64


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "oracle_csr_spmv": (None, [_I32, _I32P, _I32P, _F64P, _F64P, _F64P]),
                "oracle_csr_spmv_threads": (None, [_I32, _I32P, _I32P, _F64P, _F64P, _F64P, ctypes.c_int]),
                "oracle_row_abs_sum": (None, [_I32, _I32P, _I32P, _F64P, _F64P, _F64P]),
                "oracle_dense_matvec": (None, [_I32, _I32, _F64P, _F64P, _F64P]),
                "oracle_coo_to_csr": (None, [_I32, _I64, _I32P, _I32P, _F64P, _I32P, _I32P, _F64P]),
                "oracle_max_row_len": (_I32, [_I32, _I32P]),
                "oracle_csr_to_ell": (None, [_I32, _I32P, _I32P, _F64P, _I32, _I32P, _I32P, _F64P]),
                "oracle_ell_to_csr": (None, [_I32, _I32, _I32P, _I32P, _F64P, _I32P, _I32P, _F64P]),
                "oracle_sell_layout": (_I64, [_I32, _I32P, _I32, _I32, _I32P, _I32P, _I64P]),
                "oracle_csr_to_sell": (None, [_I32, _I32P, _I32P, _F64P, _I32, _I32P, _I64P, _I32P, _F64P]),
                "oracle_sell_to_csr": (None, [_I32, _I32, _I32P, _I32P, _I64P, _I32P, _F64P, _I32P, _I32P, _F64P]),
                "oracle_hyb_k": (_I32, [_I32, _I32P]),
                "oracle_hyb_tail_count": (_I64, [_I32, _I32P, _I32]),
                "oracle_csr_to_hyb": (None, [_I32, _I32P, _I32P, _F64P, _I32, _I32P, _I32P, _F64P, _I32P, _I32P, _F64P]),
                "oracle_hyb_to_csr": (None, [_I32, _I32, _I32P, _I32P, _F64P, _I64, _I32P, _I32P, _F64P, _I32P, _I32P, _F64P]),
                "oracle_csr5_ntiles": (_I64, [_I64, _I32, _I32]),
                "oracle_csr_to_csr5": (_I64, [_I32, _I32P, _I32P, _F64P, _I32, _I32, _I32P, _U8P, _I32P, _U8P, _I32P, _F64P, _I32P, _I32P]),
                "oracle_csr5_to_csr": (None, [_I32, _I32P, _I64, _I32, _I32, _I32P, _F64P, _I32P, _I32P, _F64P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    t = {np.int32: _I32P, np.int64: _I64P, np.float64: _F64P, np.uint8: _U8P}[a.dtype.type]
    if a.size == 0:  # never dereferenced, but keep ctypes happy
        a = np.zeros(1, dtype=a.dtype)
    return a.ctypes.data_as(t)


def _csr_arrays(a):
    return _c(a.ptr, np.int32), _c(a.idx, np.int32), _c(a.val, np.float64)


# ------------------------------------------------------------------ SpMV

def csr_spmv(a, x) -> np.ndarray:
    """y = A x (Sec. II-A) over CSR, one row at a time, in CSR order."""
    ptr, idx, val = _csr_arrays(a)
    x = _c(x, np.float64)
    y = np.empty(a.m, dtype=np.float64)
    _load().oracle_csr_spmv(a.m, _p(ptr), _p(idx), _p(val), _p(x), _p(y))
    return y


def csr_spmv_threads(a, x, nthreads: int) -> np.ndarray:
    """Same loop, rows split over nthreads (bit-identical to csr_spmv)."""
    ptr, idx, val = _csr_arrays(a)
    x = _c(x, np.float64)
    y = np.empty(a.m, dtype=np.float64)
    _load().oracle_csr_spmv_threads(a.m, _p(ptr), _p(idx), _p(val), _p(x), _p(y), nthreads)
    return y


def row_abs_sum(a, x) -> np.ndarray:
    ptr, idx, val = _csr_arrays(a)
    x = _c(x, np.float64)
    s = np.empty(a.m, dtype=np.float64)
    _load().oracle_row_abs_sum(a.m, _p(ptr), _p(idx), _p(val), _p(x), _p(s))
    return s


def fp_bound(a, x) -> np.ndarray:
    """Per-row tolerance 4 * nnz_i * 2^-53 * sum_j |a_ij x_j|."""
    return 4.0 * np.diff(a.ptr).astype(np.float64) * 2.0 ** -53 * row_abs_sum(a, x)


def dense_matvec(d, x) -> np.ndarray:
    d = _c(d, np.float64)
    x = _c(x, np.float64)
    y = np.empty(d.shape[0], dtype=np.float64)
    _load().oracle_dense_matvec(d.shape[0], d.shape[1], _p(d), _p(x), _p(y))
    return y


def coo_to_csr(m, row, col, val):
    row, col, val = _c(row, np.int32), _c(col, np.int32), _c(val, np.float64)
    ptr = np.empty(m + 1, dtype=np.int32)
    idx = np.empty(row.size, dtype=np.int32)
    v = np.empty(row.size, dtype=np.float64)
    _load().oracle_coo_to_csr(m, row.size, _p(row), _p(col), _p(val), _p(ptr), _p(idx), _p(v))
    return ptr, idx, v


# ----------------------------------------------------------------- formats

def max_row_len(a) -> int:
    return int(_load().oracle_max_row_len(a.m, _p(_c(a.ptr, np.int32))))


def to_ell(a, K: int | None = None) -> dict:
    ptr, idx, val = _csr_arrays(a)
    K = max_row_len(a) if K is None else K
    row_len = np.empty(a.m, dtype=np.int32)
    col = np.empty(K * a.m, dtype=np.int32)
    v = np.empty(K * a.m, dtype=np.float64)
    _load().oracle_csr_to_ell(a.m, _p(ptr), _p(idx), _p(val), K, _p(row_len), _p(col), _p(v))
    return {"K": K, "row_len": row_len, "col": col, "val": v}


def ell_to_csr(m, e):
    ptr = np.empty(m + 1, dtype=np.int32)
    nnz = int(e["row_len"].astype(np.int64).sum())
    idx = np.empty(nnz, dtype=np.int32)
    v = np.empty(nnz, dtype=np.float64)
    _load().oracle_ell_to_csr(m, e["K"], _p(e["row_len"]), _p(e["col"]), _p(e["val"]), _p(ptr), _p(idx), _p(v))
    return ptr, idx, v


def to_sell(a, C: int, sigma: int) -> dict:
    ptr, idx, val = _csr_arrays(a)
    lib = _load()
    perm = np.empty(a.m, dtype=np.int32)
    row_len = np.empty(a.m, dtype=np.int32)
    ns = (a.m + C - 1) // C
    slice_ptr = np.empty(ns + 1, dtype=np.int64)
    total = lib.oracle_sell_layout(a.m, _p(ptr), C, sigma, _p(perm), _p(row_len), _p(slice_ptr))
    col = np.empty(total, dtype=np.int32)
    v = np.empty(total, dtype=np.float64)
    lib.oracle_csr_to_sell(a.m, _p(ptr), _p(idx), _p(val), C, _p(perm), _p(slice_ptr), _p(col), _p(v))
    return {"C": C, "sigma": sigma, "perm": perm, "row_len": row_len, "slice_ptr": slice_ptr, "col": col, "val": v}


def sell_to_csr(m, s):
    ptr = np.empty(m + 1, dtype=np.int32)
    nnz = int(s["row_len"].astype(np.int64).sum())
    idx = np.empty(nnz, dtype=np.int32)
    v = np.empty(nnz, dtype=np.float64)
    _load().oracle_sell_to_csr(m, s["C"], _p(s["perm"]), _p(s["row_len"]), _p(s["slice_ptr"]), _p(s["col"]),
                               _p(s["val"]), _p(ptr), _p(idx), _p(v))
    return ptr, idx, v


def hyb_k(a) -> int:
    return int(_load().oracle_hyb_k(a.m, _p(_c(a.ptr, np.int32))))


def to_hyb(a, K: int | None = None) -> dict:
    ptr, idx, val = _csr_arrays(a)
    lib = _load()
    K = hyb_k(a) if K is None else K
    nt = int(lib.oracle_hyb_tail_count(a.m, _p(ptr), K))
    rl = np.empty(a.m, dtype=np.int32)
    ec = np.empty(K * a.m, dtype=np.int32)
    ev = np.empty(K * a.m, dtype=np.float64)
    cr = np.empty(nt, dtype=np.int32)
    cc = np.empty(nt, dtype=np.int32)
    cv = np.empty(nt, dtype=np.float64)
    lib.oracle_csr_to_hyb(a.m, _p(ptr), _p(idx), _p(val), K, _p(rl), _p(ec), _p(ev), _p(cr), _p(cc), _p(cv))
    return {"K": K, "row_len": rl, "col": ec, "val": ev, "coo_row": cr, "coo_col": cc, "coo_val": cv}


def hyb_to_csr(m, h):
    ptr = np.empty(m + 1, dtype=np.int32)
    nnz = int(h["row_len"].astype(np.int64).sum()) + h["coo_row"].size
    idx = np.empty(nnz, dtype=np.int32)
    v = np.empty(nnz, dtype=np.float64)
    _load().oracle_hyb_to_csr(m, h["K"], _p(h["row_len"]), _p(h["col"]), _p(h["val"]), h["coo_row"].size,
                              _p(h["coo_row"]), _p(h["coo_col"]), _p(h["coo_val"]), _p(ptr), _p(idx), _p(v))
    return ptr, idx, v


def to_csr5(a, omega: int, sigma: int) -> dict:
    ptr, idx, val = _csr_arrays(a)
    lib = _load()
    nt = int(lib.oracle_csr5_ntiles(a.nnz, omega, sigma))
    S = omega * sigma
    tile_ptr = np.empty(nt + 1, dtype=np.int32)
    flag = np.empty(nt * S, dtype=np.uint8)
    y_off = np.empty(nt * omega, dtype=np.int32)
    seg_off = np.empty(nt * omega, dtype=np.uint8)
    tidx = np.empty(nt * S, dtype=np.int32)
    tval = np.empty(nt * S, dtype=np.float64)
    eptr = np.empty(nt + 1, dtype=np.int32)
    args = (a.m, _p(ptr), _p(idx), _p(val), omega, sigma, _p(tile_ptr), _p(flag), _p(y_off), _p(seg_off),
            _p(tidx), _p(tval), _p(eptr))
    ne = int(lib.oracle_csr_to_csr5(*args, None))
    erows = np.empty(ne, dtype=np.int32)
    lib.oracle_csr_to_csr5(*args, _p(erows))
    return {"omega": omega, "sigma": sigma, "ntiles": nt, "ptr": ptr.copy(), "tile_ptr": tile_ptr, "bit_flag": flag,
            "y_off": y_off, "seg_off": seg_off, "idx": tidx, "val": tval, "empty_ptr": eptr, "empty_rows": erows}


def csr5_to_csr(m, nnz, t):
    ptr = np.empty(m + 1, dtype=np.int32)
    idx = np.empty(nnz, dtype=np.int32)
    v = np.empty(nnz, dtype=np.float64)
    _load().oracle_csr5_to_csr(m, _p(t["ptr"]), nnz, t["omega"], t["sigma"], _p(t["idx"]), _p(t["val"]),
                               _p(ptr), _p(idx), _p(v))
    return ptr, idx, v
