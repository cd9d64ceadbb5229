"""ctypes binding of libspmv_gb300.so (the C ABI declared in include/spmv.h).

Argument marshalling only: every step of every call runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors (device memory); the stream is
torch's current CUDA stream unless one is given.  Loading fails loudly when the
library has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspmv_gb300.so")

SPMV_CSR, SPMV_CSR5, SPMV_ELL, SPMV_SELL, SPMV_HYB = 0, 1, 2, 3, 4
FORMATS = ("CSR", "CSR5", "ELL", "SELL", "HYB")
NUM_FEATURES = 16
MLP_PARAMS = 5573
SPMV_HYB_K_NONE = -1
SPMV_SELL_SIGMA_ALL = -1
SPMV_BATCH_ONE_LAUNCH = 1

STATUS = {0: "OK", -1: "INVALID_ARG", -2: "INDEX_OVERFLOW", -3: "TOO_LARGE", -4: "CUDA", -5: "NO_MODEL",
          -6: "ALLOC", -7: "WRONG_FORMAT"}


class SpmvError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name} ({detail})")


class spmv_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("ptr", ctypes.c_void_p), ("idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class spmv_params(ctypes.Structure):
    _fields_ = [("sell_C", ctypes.c_int32), ("sell_sigma", ctypes.c_int32), ("csr5_omega", ctypes.c_int32),
                ("csr5_sigma", ctypes.c_int32), ("csr_block_nnz", ctypes.c_int32), ("hyb_k", ctypes.c_int32),
                ("sell_panel_cols", ctypes.c_int32), ("max_bytes", ctypes.c_int64)]


class spmv_info(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("stored_slots", ctypes.c_int64), ("params", spmv_params),
                ("aux", ctypes.c_int64 * 4)]


_lib = None

_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_F = ctypes.c_float
_SIGS = {
    "spmv_version": (ctypes.c_int, []),
    "spmv_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "spmv_last_error": (ctypes.c_char_p, []),
    "spmv_convert": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(spmv_csr), ctypes.POINTER(spmv_params), _VP,
                                    ctypes.POINTER(_VP)]),
    "spmv_run": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "spmv_to_csr": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "spmv_handle_info": (ctypes.c_int, [_VP, ctypes.POINTER(spmv_info)]),
    "spmv_handle_array": (ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(_I32)]),
    "spmv_free": (None, [_VP]),
    "spmv_features": (ctypes.c_int, [ctypes.POINTER(spmv_csr), _VP, _VP]),
    "spmv_model_create": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "spmv_model_free": (None, [_VP]),
    "spmv_model_set_max_bytes": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "spmv_select_async": (ctypes.c_int, [ctypes.POINTER(spmv_csr), _VP, _VP, _VP, _VP]),
    "spmv_select": (ctypes.c_int, [ctypes.POINTER(spmv_csr), _VP, _VP, ctypes.POINTER(ctypes.c_int)]),
    "spmv_mlp_scale": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _VP]),
    "spmv_mlp_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _VP, _VP]),
    "spmv_mlp_adam": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _I32, _F, _F, _F, _F, _VP]),
    "spmv_mlp_train": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I32, _I32, _I32, _F, _F, _F, _F, _VP, _VP]),
    "spmv_mlp_forward": (ctypes.c_int, [_VP, _VP, _I32, _VP, _VP, _VP]),
    "spmv_host_io_create": (ctypes.c_int, [_VP, ctypes.POINTER(_VP)]),
    "spmv_run_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "spmv_host_io_sync": (ctypes.c_int, [_VP]),
    "spmv_host_io_free": (None, [_VP]),
    "spmv_batch_build": (ctypes.c_int, [ctypes.POINTER(_VP), _I32, _VP, ctypes.POINTER(_VP)]),
    "spmv_batch_build_ex": (ctypes.c_int, [ctypes.POINTER(_VP), _I32, _I32, _VP, ctypes.POINTER(_VP)]),
    "spmv_batch_launches": (ctypes.c_int, [_VP, ctypes.POINTER(_I32)]),
    "spmv_batch_run": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    "spmv_batch_run_separate": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    "spmv_batch_free": (None, [_VP]),
    "spmv_csr_run_noalloc": (ctypes.c_int, [ctypes.POINTER(spmv_csr), _VP, _VP, _VP]),
    "spmv_debug_fail_alloc": (None, [_I32]),
    "spmv_debug_features_cluster": (None, [_I32]),
}
EXPORTED = tuple(_SIGS)


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it was not built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != 0:
        detail = lib().spmv_last_error()
        raise SpmvError(status, where, detail.decode() if detail else "")
