"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

Only inputs are made here (CSR patterns, values, dense vectors, workload
parameters); nothing here multiplies, converts or selects.  The heavy lifting
is in ``synth.c`` (counter-based generator, pthreads), compiled on first use
with the system C compiler so it works on any host architecture.

Workload recipes (all square, FP64 values, int32 indices, columns ascending
within a row):

* ``laplacian2d(nx, ny)``: 5-point Laplacian, 4 on the diagonal, -1 off it.
* ``powerlaw(n, ...)``: row lengths ceil(X), X a Pareto law with density
  proportional to x^-alpha truncated to [xmin, xmax]; columns uniform and
  distinct per row (duplicates resampled); values N(0,1).
* ``stencil(kind, nx, ny, nz)``: 2D 5/9-point or 3D 7/27-point stencils,
  values N(0,1) off the diagonal and 1 + sum|off-diagonal| on it.
* ``banded``, ``blockdiag``, ``uniform_random``: the other corpus families.
* ``vector(n, seed)``: x uniform in [-1, 1).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

NTHREADS = max(1, len(os.sched_getaffinity(0)))


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, -O2, no arch flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            f64p = ctypes.POINTER(ctypes.c_double)
            i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            cint = ctypes.c_int
            sig = {
                "synth_powerlaw_lengths": (i64, [i32, f64, f64, f64, i32, i32, u64, i32p]),
                "synth_uniform_lengths": (i64, [i32, i32, i32, u64, i32p]),
                "synth_lengths_to_ptr": (i64, [i32, i32p, i32p]),
                "synth_fill_random_cols": (None, [i32, i32, i32p, u64, i32p, cint]),
                "synth_fill_normal": (None, [i64, u64, f64p, cint]),
                "synth_fill_uniform": (None, [i64, u64, f64, f64, f64p, cint]),
                "synth_fill_int": (None, [i64, u64, i64, i64, f64p, cint]),
                "synth_stencil_lengths": (None, [cint, cint, cint, cint, i32p, cint]),
                "synth_stencil_cols": (None, [cint, cint, cint, cint, i32p, i32p, cint]),
                "synth_diag_dominant": (None, [i32, i32p, i32p, f64p]),
                "synth_band_lengths": (None, [i32, i32, i32p]),
                "synth_band_cols": (None, [i32, i32, i32p, i32p]),
                "synth_blockdiag_lengths": (None, [i32, i32, i32p]),
                "synth_blockdiag_cols": (None, [i32, i32, i32p, i32p]),
                "synth_scalar_u01": (f64, [u64, u64, u64]),
                "synth_scalar_u64": (u64, [u64, u64, u64]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclasses.dataclass
class CSR:
    """A host CSR matrix: ptr int32[m+1], idx int32[nnz], val float64[nnz]."""

    m: int
    n: int
    ptr: np.ndarray
    idx: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.ptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.ptr)


U64 = (1 << 64) - 1


def seed_of(config: int, index: int) -> int:
    """64-bit seed of matrix `index` of workload `config` (a hash of both)."""
    return int(_load().synth_scalar_u64(0x5EED5EED, config, index)) & U64


def u01(seed: int, stream: int, ctr: int) -> float:
    return float(_load().synth_scalar_u01(seed & U64, stream & U64, ctr & U64))


def _ptr_from_lengths(lengths: np.ndarray) -> np.ndarray:
    m = lengths.shape[0]
    ptr = np.empty(m + 1, dtype=np.int32)
    tot = _load().synth_lengths_to_ptr(m, _p32(lengths), _p32(ptr))
    if tot < 0:
        raise OverflowError("matrix has more than 2^31-1 nonzeros")
    return ptr


def normal(nnz: int, seed: int) -> np.ndarray:
    out = np.empty(nnz, dtype=np.float64)
    _load().synth_fill_normal(nnz, seed & U64, _p64(out), NTHREADS)
    return out


def vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Dense vector, uniform in [lo, hi)."""
    out = np.empty(n, dtype=np.float64)
    _load().synth_fill_uniform(n, seed & U64, lo, hi, _p64(out), NTHREADS)
    return out


def integers(nnz: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """Integer values uniform in {lo..hi}, as float64."""
    out = np.empty(nnz, dtype=np.float64)
    _load().synth_fill_int(nnz, seed & U64, lo, hi, _p64(out), NTHREADS)
    return out


def from_lengths_random_cols(lengths: np.ndarray, n_cols: int, seed: int, name: str = "") -> CSR:
    lengths = np.ascontiguousarray(lengths, dtype=np.int32)
    m = lengths.shape[0]
    ptr = _ptr_from_lengths(lengths)
    idx = np.empty(int(ptr[-1]), dtype=np.int32)
    _load().synth_fill_random_cols(m, n_cols, _p32(ptr), (seed ^ 0xC015) & U64, _p32(idx), NTHREADS)
    val = normal(int(ptr[-1]), seed ^ 0x5A15)
    return CSR(m, n_cols, ptr, idx, val, name)


def powerlaw_lengths(m: int, seed: int, alpha: float = 2.1, xmin: float = 1.0, xmax: float = 5000.0,
                     lmin: int = 1, lmax: int = 5000) -> np.ndarray:
    out = np.empty(m, dtype=np.int32)
    _load().synth_powerlaw_lengths(m, alpha, xmin, xmax, lmin, lmax, seed & U64, _p32(out))
    return out


def powerlaw(n: int, seed: int, alpha: float = 2.1, xmin: float = 1.0, xmax: float = 5000.0,
             lmin: int = 1, lmax: int = 5000, name: str = "powerlaw") -> CSR:
    lmax = min(lmax, n)
    lengths = powerlaw_lengths(n, seed, alpha, xmin, min(xmax, float(lmax)), lmin, lmax)
    return from_lengths_random_cols(lengths, n, seed, name)


def uniform_random(n: int, r: int, seed: int, name: str = "uniform") -> CSR:
    """Every row holds r distinct uniform columns."""
    r = min(r, n)
    return from_lengths_random_cols(np.full(n, r, dtype=np.int32), n, seed, name)


def uniform_lengths(m: int, lo: int, hi: int, seed: int) -> np.ndarray:
    out = np.empty(m, dtype=np.int32)
    _load().synth_uniform_lengths(m, lo, hi, seed & U64, _p32(out))
    return out


STENCIL_5PT_2D, STENCIL_9PT_2D, STENCIL_7PT_3D, STENCIL_27PT_3D = 0, 1, 2, 3


def stencil_pattern(kind: int, nx: int, ny: int, nz: int = 1):
    lib = _load()
    m = nx * ny * nz
    ptr = np.zeros(m + 1, dtype=np.int32)
    lib.synth_stencil_lengths(kind, nx, ny, nz, _p32(ptr), NTHREADS)
    lengths = ptr[1:].copy()
    ptr = _ptr_from_lengths(lengths)
    idx = np.empty(int(ptr[-1]), dtype=np.int32)
    lib.synth_stencil_cols(kind, nx, ny, nz, _p32(ptr), _p32(idx), NTHREADS)
    return ptr, idx


def stencil(kind: int, nx: int, ny: int, nz: int = 1, seed: int = 0, name: str = "stencil") -> CSR:
    """Stencil pattern; N(0,1) off-diagonal, diagonal 1 + sum|off-diagonal|."""
    ptr, idx = stencil_pattern(kind, nx, ny, nz)
    val = normal(int(ptr[-1]), seed)
    m = nx * ny * nz
    _load().synth_diag_dominant(m, _p32(ptr), _p32(idx), _p64(val))
    return CSR(m, m, ptr, idx, val, name)


def laplacian2d(nx: int, ny: int) -> CSR:
    """2D 5-point Laplacian: 4 on the diagonal, -1 for each in-grid neighbour."""
    ptr, idx = stencil_pattern(STENCIL_5PT_2D, nx, ny, 1)
    m = nx * ny
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(ptr))
    val = np.where(idx == rows, 4.0, -1.0)
    return CSR(m, m, ptr, idx, val, f"laplacian2d_{nx}x{ny}")


def banded(n: int, bw: int, seed: int, name: str = "banded") -> CSR:
    lib = _load()
    lengths = np.empty(n, dtype=np.int32)
    lib.synth_band_lengths(n, bw, _p32(lengths))
    ptr = _ptr_from_lengths(lengths)
    idx = np.empty(int(ptr[-1]), dtype=np.int32)
    lib.synth_band_cols(n, bw, _p32(ptr), _p32(idx))
    return CSR(n, n, ptr, idx, normal(int(ptr[-1]), seed), name)


def blockdiag(n: int, b: int, seed: int, name: str = "blockdiag") -> CSR:
    lib = _load()
    lengths = np.empty(n, dtype=np.int32)
    lib.synth_blockdiag_lengths(n, b, _p32(lengths))
    ptr = _ptr_from_lengths(lengths)
    idx = np.empty(int(ptr[-1]), dtype=np.int32)
    lib.synth_blockdiag_cols(n, b, _p32(ptr), _p32(idx))
    return CSR(n, n, ptr, idx, normal(int(ptr[-1]), seed), name)


def with_integer_values(a: CSR, seed: int, lo: int = -8, hi: int = 8) -> CSR:
    """Same pattern, small integer values (every summation order is exact)."""
    return CSR(a.m, a.n, a.ptr, a.idx, integers(a.nnz, seed, lo, hi), a.name + "_int")


def from_dense(d: np.ndarray, name: str = "dense") -> CSR:
    """CSR of the nonzero pattern of a dense array (explicit zeros dropped)."""
    m, n = d.shape
    rows, cols = np.nonzero(d)
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(ptr, rows + 1, 1)
    ptr = np.cumsum(ptr).astype(np.int32)
    return CSR(m, n, ptr, cols.astype(np.int32), d[rows, cols].astype(np.float64), name)


def tiny_random(m: int, n: int, density: float, seed: int, integer: bool = False) -> CSR:
    """Small random matrix for brute-force tests (Bernoulli pattern)."""
    mask = np.array([u01(seed, 7, k) < density for k in range(m * n)], dtype=bool).reshape(m, n)
    d = np.zeros((m, n))
    nz = int(mask.sum())
    vals = integers(nz, seed, -9, 9) if integer else normal(nz, seed)
    vals[vals == 0] = 1.0
    d[mask] = vals
    return from_dense(d, f"tiny_{m}x{n}")


# ----------------------------------------------------------- workload specs

# Workload 5b: x_min that gives E[ceil(X)] close to 12 for alpha = 2.1 on [xmin, 1e5].
GRAPH_XMIN = 1.56


def config1() -> CSR:
    """2D 5-point Laplacian on a 64 x 64 grid: n = 4096, nnz = 20224."""
    return laplacian2d(64, 64)


def config2(seed: int | None = None) -> CSR:
    """n = 2e6, power-law row lengths (alpha 2.1 on [1, 5000]), uniform columns, N(0,1) values."""
    s = seed_of(2, 0) if seed is None else seed
    return powerlaw(2_000_000, s, name="powerlaw_2e6")


def config5_stencil(side: int = 224) -> CSR:
    """3D 27-point stencil on side^3 (224^3: n = 11,239,424, nnz = 300,763,000)."""
    return stencil(STENCIL_27PT_3D, side, side, side, seed_of(5, 0), name=f"stencil27_{side}^3")


def config5_graph(n: int = 20_000_000) -> CSR:
    """Power-law graph: alpha 2.1, mean about 12 nonzeros per row, at most 1e5."""
    return powerlaw(n, seed_of(5, 1), xmin=GRAPH_XMIN, xmax=1e5, lmax=100_000, name=f"graph_{n}")


CORPUS_FAMILIES = ("banded", "stencil", "blockdiag", "uniform", "powerlaw")


def corpus_spec(i: int, n_lo: float = 1e3, n_hi: float = 5e6) -> dict:
    """Parameters of corpus matrix i: n log-uniform in [n_lo, n_hi], family uniform over five."""
    s = seed_of(3, i)
    n = int(round(10 ** (math.log10(n_lo) + u01(s, 1, 0) * (math.log10(n_hi) - math.log10(n_lo)))))
    fam = CORPUS_FAMILIES[min(4, int(u01(s, 1, 1) * 5))]
    spec = {"index": i, "seed": s, "family": fam, "n": n}
    if fam == "banded":
        spec["bw"] = 1 + int(u01(s, 1, 2) * 64)
    elif fam == "stencil":
        kind = min(3, int(u01(s, 1, 2) * 4))
        spec["kind"] = kind
        if kind < 2:
            side = max(2, int(round(math.sqrt(n))))
            spec["grid"] = (side, side, 1)
        else:
            side = max(2, int(round(n ** (1.0 / 3.0))))
            spec["grid"] = (side, side, side)
        spec["n"] = spec["grid"][0] * spec["grid"][1] * spec["grid"][2]
    elif fam == "blockdiag":
        spec["block"] = 4 + int(u01(s, 1, 2) * 61)
    elif fam == "uniform":
        spec["r"] = 2 + int(u01(s, 1, 2) * 63)
    return spec


def corpus_matrix(i: int, **kw) -> CSR:
    sp = corpus_spec(i, **kw)
    s, n, fam = sp["seed"], sp["n"], sp["family"]
    name = f"corpus{i}_{fam}"
    if fam == "banded":
        return banded(n, sp["bw"], s, name)
    if fam == "stencil":
        nx, ny, nz = sp["grid"]
        return stencil(sp["kind"], nx, ny, nz, s, name)
    if fam == "blockdiag":
        return blockdiag(n, sp["block"], s, name)
    if fam == "uniform":
        return uniform_random(n, sp["r"], s, name)
    return powerlaw(n, s, name=name)


def batch_spec(j: int, r_lo: float = 1e3, r_hi: float = 2e5) -> dict:
    """Matrix j of the batched workload: rows log-uniform, lengths in [3, 200]."""
    s = seed_of(4, j)
    n = int(round(math.exp(math.log(r_lo) + u01(s, 1, 0) * (math.log(r_hi) - math.log(r_lo)))))
    law = "uniform" if u01(s, 1, 1) < 0.5 else "powerlaw"
    return {"index": j, "seed": s, "n": n, "law": law}


def batch_matrix(j: int, **kw) -> CSR:
    sp = batch_spec(j, **kw)
    n, s = sp["n"], sp["seed"]
    if sp["law"] == "uniform":
        lengths = uniform_lengths(n, 3, min(200, n), s)
    else:
        lengths = powerlaw_lengths(n, s, xmin=3.0, xmax=200.0, lmin=3, lmax=min(200, n))
    return from_lengths_random_cols(lengths, n, s, f"batch{j}_{sp['law']}")
