"""Gather-ceiling probe of the benchmark (libspmv_probe.so, built from
``gather.cu`` beside this file).  A measurement aid, not part of the
library's C ABI: the benchmark times it on a matrix's own index stream
beside the product."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspmv_probe.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1805_11938_gb300.build first")
        L = ctypes.CDLL(LIB_PATH)
        L.spmv_probe_partials.restype = ctypes.c_int
        L.spmv_probe_partials.argtypes = []
        L.spmv_probe_gather.restype = ctypes.c_int
        L.spmv_probe_gather.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        _lib = L
    return _lib


def partials() -> int:
    n = lib().spmv_probe_partials()
    if n <= 0:
        raise RuntimeError("spmv_probe_partials: no CUDA device")
    return n


def gather(csr, x, partial=None, stream=None):
    """Partial sums of val[k] * x[idx[k]] over the CSR's entries (csr: a
    DeviceCSR); their sum is the total."""
    import torch

    if partial is None:
        partial = torch.empty(partials(), dtype=torch.float64, device=x.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().spmv_probe_gather(ctypes.c_void_p(csr.idx.data_ptr()), ctypes.c_void_p(csr.val.data_ptr()),
                                 int(csr.nnz), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(partial.data_ptr()),
                                 int(partial.numel()), ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"spmv_probe_gather failed ({rc})")
    return partial
