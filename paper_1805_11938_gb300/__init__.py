"""GB300 (sm_103a) FP64 SpMV in the five representations of arXiv:1805.11938.

Thin Python layer over the C ABI (include/spmv.h, libspmv_gb300.so).  Device
memory and streams come from PyTorch; every computation runs in the library's
CUDA kernels.  The functions keep the C names:

    h = spmv_convert(SPMV_SELL, DeviceCSR.from_host(a), {"sell_C": 64})
    y = spmv_run(h, x)                 # y = A x on the current stream
    ptr, idx, val = spmv_to_csr(h)     # exact round trip
    f = spmv_features(csr)             # 16 float32 features
    fmt = spmv_select(csr, model)      # learned format choice
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _abi
from ._abi import (FORMATS, MLP_PARAMS, NUM_FEATURES, SPMV_CSR, SPMV_CSR5, SPMV_ELL, SPMV_HYB, SPMV_HYB_K_NONE,  # noqa: F401
                   SPMV_SELL, SPMV_SELL_SIGMA_ALL, SpmvError, check, lib)

__all__ = [
    "FORMATS", "SPMV_CSR", "SPMV_CSR5", "SPMV_ELL", "SPMV_SELL", "SPMV_HYB", "SPMV_HYB_K_NONE", "SPMV_SELL_SIGMA_ALL",
    "SpmvError", "DeviceCSR", "Handle", "Model", "Batch", "spmv_convert", "spmv_run", "spmv_to_csr",
    "spmv_features", "spmv_select", "spmv_select_async", "spmv_mlp_scale", "spmv_mlp_loss_grad", "spmv_mlp_adam",
    "spmv_mlp_train", "spmv_mlp_forward", "spmv_batch_build", "spmv_batch_run", "spmv_batch_run_separate",
    "spmv_csr_run_noalloc", "spmv_debug_fail_alloc", "spmv_debug_features_cluster", "lib", "HostIO",
    "spmv_host_io_create", "spmv_run_host",
]


def _torch():
    import torch

    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


_cudart = None


def _memcpy_d2d(dst_ptr: int, src_ptr: int, nbytes: int) -> None:
    """Plain cudaMemcpy (device to device) used to read handle arrays."""
    global _cudart
    if _cudart is None:
        for cand in ("libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
            try:
                _cudart = ctypes.CDLL(cand)
                break
            except OSError:
                continue
        if _cudart is None:
            raise RuntimeError("libcudart not found")
        _cudart.cudaMemcpy.restype = ctypes.c_int
        _cudart.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    if nbytes:
        rc = _cudart.cudaMemcpy(ctypes.c_void_p(dst_ptr), ctypes.c_void_p(src_ptr), nbytes, 3)
        if rc != 0:
            raise RuntimeError(f"cudaMemcpy failed ({rc})")


class DeviceCSR:
    """CSR arrays resident on the GPU (int32 ptr/idx, float64 val)."""

    def __init__(self, m: int, n: int, ptr, idx, val):
        self.m, self.n = int(m), int(n)
        self.ptr, self.idx, self.val = ptr, idx, val
        self.nnz = int(idx.numel())
        self._c = _abi.spmv_csr(self.m, self.n, self.nnz, ptr.data_ptr(), idx.data_ptr() if self.nnz else None,
                                val.data_ptr() if self.nnz else None)

    @classmethod
    def from_host(cls, a, device: str = "cuda") -> "DeviceCSR":
        torch = _torch()
        ptr = torch.as_tensor(np.ascontiguousarray(a.ptr, dtype=np.int32)).to(device)
        idx = torch.as_tensor(np.ascontiguousarray(a.idx, dtype=np.int32)).to(device)
        val = torch.as_tensor(np.ascontiguousarray(a.val, dtype=np.float64)).to(device)
        return cls(a.m, a.n, ptr, idx, val)

    @property
    def c(self):
        return self._c


def _params(p) -> _abi.spmv_params | None:
    if p is None:
        return None
    if isinstance(p, _abi.spmv_params):
        return p
    out = _abi.spmv_params()
    for k, v in p.items():
        setattr(out, k, int(v))
    return out


class Handle:
    """A matrix converted to one format; owns its device buffers."""

    def __init__(self, ptr: int, csr_shape):
        self._h = ctypes.c_void_p(ptr)
        self.m, self.n = csr_shape

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _abi._lib is not None:
            _abi._lib.spmv_free(self._h)
            self._h = None

    def free(self):
        self.__del__()

    @property
    def raw(self):
        return self._h

    def info(self) -> dict:
        inf = _abi.spmv_info()
        check(lib().spmv_handle_info(self._h, ctypes.byref(inf)), "spmv_handle_info")
        p = inf.params
        return {"fmt": inf.fmt, "format": FORMATS[inf.fmt], "m": inf.m, "n": inf.n, "nnz": inf.nnz,
                "device_bytes": inf.device_bytes, "stored_slots": inf.stored_slots, "aux": list(inf.aux),
                "params": {k: getattr(p, k) for k, _ in _abi.spmv_params._fields_}}

    def array(self, name: str):
        """A copy (torch tensor on the GPU) of one of the handle's arrays."""
        torch = _torch()
        ptr = ctypes.c_void_p()
        cnt = ctypes.c_int64()
        eb = ctypes.c_int32()
        check(lib().spmv_handle_array(self._h, name.encode(), ctypes.byref(ptr), ctypes.byref(cnt), ctypes.byref(eb)),
              f"spmv_handle_array({name})")
        dt = {1: torch.uint8, 4: torch.int32, 8: torch.int64, 16: torch.int32}[eb.value]
        n = cnt.value * (4 if eb.value == 16 else 1)
        out = torch.empty(n, dtype=dt, device="cuda")
        torch.cuda.synchronize()
        _memcpy_d2d(out.data_ptr(), ptr.value or 0, cnt.value * eb.value)
        return out

    def run(self, x, y=None, stream=None):
        return spmv_run(self, x, y, stream)


def spmv_convert(fmt: int, csr: DeviceCSR, params=None, stream=None) -> Handle:
    out = ctypes.c_void_p()
    p = _params(params)
    check(lib().spmv_convert(int(fmt), ctypes.byref(csr.c), ctypes.byref(p) if p is not None else None,
                             _stream(stream), ctypes.byref(out)), f"spmv_convert({FORMATS[int(fmt)] if 0 <= int(fmt) < 5 else fmt})")
    return Handle(out.value, (csr.m, csr.n))


def spmv_run(h: Handle, x, y=None, stream=None):
    torch = _torch()
    if y is None:
        y = torch.empty(h.m, dtype=torch.float64, device=x.device)
    check(lib().spmv_run(h.raw, _vp(x), _vp(y), _stream(stream)), "spmv_run")
    return y


def spmv_to_csr(h: Handle, stream=None):
    torch = _torch()
    info = h.info()
    ptr = torch.empty(h.m + 1, dtype=torch.int32, device="cuda")
    idx = torch.empty(max(info["nnz"], 0), dtype=torch.int32, device="cuda")
    val = torch.empty(max(info["nnz"], 0), dtype=torch.float64, device="cuda")
    check(lib().spmv_to_csr(h.raw, _vp(ptr), _vp(idx) if info["nnz"] else None, _vp(val) if info["nnz"] else None,
                            _stream(stream)), "spmv_to_csr")
    return ptr, idx, val


def spmv_features(csr: DeviceCSR, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = torch.empty(NUM_FEATURES, dtype=torch.float32, device="cuda")
    check(lib().spmv_features(ctypes.byref(csr.c), _vp(out), _stream(stream)), "spmv_features")
    return out


class Model:
    """A trained selector: network parameters plus the feature scaling table."""

    def __init__(self, params, lo, hi):
        p = np.ascontiguousarray(params, dtype=np.float32)
        l = np.ascontiguousarray(lo, dtype=np.float32)
        h = np.ascontiguousarray(hi, dtype=np.float32)
        if p.size != MLP_PARAMS or l.size != NUM_FEATURES or h.size != NUM_FEATURES:
            raise ValueError("model needs 5573 parameters and 16 lo/hi values")
        self.params, self.lo, self.hi = p, l, h
        out = ctypes.c_void_p()
        check(lib().spmv_model_create(p.ctypes.data_as(ctypes.c_void_p), l.ctypes.data_as(ctypes.c_void_p),
                                      h.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)), "spmv_model_create")
        self._m = out

    def __del__(self):
        if getattr(self, "_m", None) and self._m.value and _abi._lib is not None:
            _abi._lib.spmv_model_free(self._m)
            self._m = None

    @property
    def raw(self):
        return self._m

    def set_max_bytes(self, max_bytes: int) -> None:
        """Footprint cap for selection: spmv_select never names ELL above it."""
        check(lib().spmv_model_set_max_bytes(self._m, int(max_bytes)), "spmv_model_set_max_bytes")

    @classmethod
    def load(cls, path: str) -> "Model":
        import json

        with open(path) as f:
            d = json.load(f)
        return cls(np.array(d["params"], np.float32), np.array(d["lo"], np.float32), np.array(d["hi"], np.float32))


def spmv_select(csr: DeviceCSR, model: Model | None, stream=None) -> int:
    out = ctypes.c_int()
    check(lib().spmv_select(ctypes.byref(csr.c), model.raw if model is not None else None, _stream(stream),
                            ctypes.byref(out)), "spmv_select")
    return out.value


def spmv_select_async(csr: DeviceCSR, model: Model, fmt_out, logits_out=None, stream=None):
    check(lib().spmv_select_async(ctypes.byref(csr.c), model.raw if model is not None else None, _vp(fmt_out),
                                  _vp(logits_out), _stream(stream)), "spmv_select_async")
    return fmt_out


def spmv_mlp_scale(feat, lo, hi, stream=None):
    torch = _torch()
    B = feat.shape[0]
    X = torch.empty((B, NUM_FEATURES), dtype=torch.float32, device="cuda")
    check(lib().spmv_mlp_scale(_vp(feat), _vp(lo), _vp(hi), B, _vp(X), _stream(stream)), "spmv_mlp_scale")
    return X


def spmv_mlp_loss_grad(theta, X, labels, stream=None):
    torch = _torch()
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    check(lib().spmv_mlp_loss_grad(_vp(theta), _vp(X), _vp(labels), X.shape[0], _vp(g), _vp(loss), _stream(stream)),
          "spmv_mlp_loss_grad")
    return loss, g


def spmv_mlp_adam(theta, grad, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(lib().spmv_mlp_adam(_vp(theta), _vp(grad), _vp(m), _vp(v), theta.numel(), t, lr, beta1, beta2, eps,
                              _stream(stream)), "spmv_mlp_adam")


def spmv_mlp_train(theta, m, v, X, labels, steps: int, t0: int = 0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   stream=None):
    torch = _torch()
    hist = torch.empty(max(steps, 1), dtype=torch.float32, device="cuda")
    check(lib().spmv_mlp_train(_vp(theta), _vp(m), _vp(v), _vp(X), _vp(labels), X.shape[0], steps, t0, lr, beta1,
                               beta2, eps, _vp(hist), _stream(stream)), "spmv_mlp_train")
    return hist


def spmv_mlp_forward(theta, X, stream=None):
    torch = _torch()
    B = X.shape[0]
    logits = torch.empty((B, 5), dtype=torch.float32, device="cuda")
    pred = torch.empty(B, dtype=torch.int32, device="cuda")
    check(lib().spmv_mlp_forward(_vp(theta), _vp(X), B, _vp(logits), _vp(pred), _stream(stream)), "spmv_mlp_forward")
    return logits, pred


class HostIO:
    """Products of one handle with x and y in host memory (include/spmv.h,
    spmv_run_host): two device staging pairs used in turn and two copy
    streams, so one call's copies overlap the neighbouring calls' products."""

    def __init__(self, h: Handle):
        self.h = h  # the handle must outlive the io
        out = ctypes.c_void_p()
        check(lib().spmv_host_io_create(h.raw, ctypes.byref(out)), "spmv_host_io_create")
        self._io = out

    def run(self, x_host, y_host, stream=None, done=None):
        """y_host = A x_host (float64 CPU tensors, pinned for asynchronous copies).
        Returns at once; y_host holds the result after sync(), or once the
        torch.cuda.Event `done` has completed."""
        torch = _torch()
        for t, n, what in ((x_host, self.h.n, "x_host"), (y_host, self.h.m, "y_host")):
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
                raise ValueError(f"{what} must be a contiguous float64 CPU tensor of {n} elements")
        if done is not None and not done.cuda_event:
            done.record()  # torch creates its events at their first record
        ev = ctypes.c_void_p(done.cuda_event) if done is not None else None
        check(lib().spmv_run_host(self._io, _vp(x_host), _vp(y_host), _stream(stream), ev), "spmv_run_host")

    def sync(self):
        check(lib().spmv_host_io_sync(self._io), "spmv_host_io_sync")

    def __del__(self):
        if getattr(self, "_io", None) and self._io.value and _abi._lib is not None:
            _abi._lib.spmv_host_io_free(self._io)
            self._io = None


def spmv_host_io_create(h: Handle) -> HostIO:
    return HostIO(h)


def spmv_run_host(io: HostIO, x_host, y_host, stream=None, done=None):
    io.run(x_host, y_host, stream, done)


class Batch:
    """Several handles multiplied in one persistent launch replayed from a CUDA graph."""

    def __init__(self, handles, stream=None, one_launch: bool = False):
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.raw.value for h in self.handles])
        out = ctypes.c_void_p()
        flags = _abi.SPMV_BATCH_ONE_LAUNCH if one_launch else 0
        check(lib().spmv_batch_build_ex(arr, len(self.handles), flags, _stream(stream), ctypes.byref(out)),
              "spmv_batch_build_ex")
        self._b = out

    def launches(self) -> int:
        """Kernels one replay runs."""
        n = ctypes.c_int32()
        check(lib().spmv_batch_launches(self._b, ctypes.byref(n)), "spmv_batch_launches")
        return n.value

    def __del__(self):
        if getattr(self, "_b", None) and self._b.value and _abi._lib is not None:
            _abi._lib.spmv_batch_free(self._b)
            self._b = None

    def _tables(self, xs, ys):
        n = len(self.handles)
        xa = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        return xa, ya

    def run(self, xs, ys, stream=None):
        xa, ya = self._tables(xs, ys)
        check(lib().spmv_batch_run(self._b, xa, ya, _stream(stream)), "spmv_batch_run")

    def run_separate(self, xs, ys, stream=None):
        xa, ya = self._tables(xs, ys)
        check(lib().spmv_batch_run_separate(self._b, xa, ya, _stream(stream)), "spmv_batch_run_separate")


def spmv_batch_build(handles, stream=None, one_launch: bool = False) -> Batch:
    return Batch(handles, stream, one_launch)


def spmv_batch_run(b: Batch, xs, ys, stream=None):
    b.run(xs, ys, stream)


def spmv_batch_run_separate(b: Batch, xs, ys, stream=None):
    b.run_separate(xs, ys, stream)


def spmv_csr_run_noalloc(csr: DeviceCSR, x, y=None, stream=None):
    """y = A x from the caller's CSR with no device allocation (see include/spmv.h)."""
    torch = _torch()
    if y is None:
        y = torch.empty(csr.m, dtype=torch.float64, device=x.device)
    check(lib().spmv_csr_run_noalloc(ctypes.byref(csr.c), _vp(x), _vp(y), _stream(stream)), "spmv_csr_run_noalloc")
    return y


def spmv_debug_fail_alloc(k: int) -> None:
    lib().spmv_debug_fail_alloc(int(k))


def spmv_debug_features_cluster(ctas: int) -> None:
    lib().spmv_debug_features_cluster(int(ctas))


# the selector trained on single-product times (spmv_select's default use), and
# the one trained on throughput times, which picks formats inside a batch
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "selector_mlp.json")
MODEL_BATCH_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "selector_mlp_batch.json")
