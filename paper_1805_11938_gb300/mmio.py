"""Matrix Market input (the SuiteSparse collection's file format) to the host CSR
the library converts from.

Reads the coordinate format with real, integer or pattern fields and general,
symmetric or skew-symmetric symmetry (1-based indices; pattern entries get the
value 1.0; a symmetric file's off-diagonal entry (i, j) also gives (j, i),
negated for skew-symmetric).  Entries keep the file's order within each row;
duplicates are kept (the products sum them, as for any CSR input).  Complex
and array-format files are refused.

    from paper_1805_11938_gb300.mmio import read_mtx
    a = read_mtx("matrix.mtx")          # .m .n .ptr .idx .val (int32/float64 numpy)
    d = DeviceCSR.from_host(a)
"""
from __future__ import annotations

import gzip
from dataclasses import dataclass

import numpy as np


@dataclass
class HostCSR:
    m: int
    n: int
    ptr: np.ndarray
    idx: np.ndarray
    val: np.ndarray
    name: str = "mtx"

    @property
    def nnz(self) -> int:
        return int(self.idx.size)


def _open(path):
    return gzip.open(path, "rt") if str(path).endswith(".gz") else open(path, "r")


def read_mtx(path) -> HostCSR:
    with _open(path) as f:
        header = f.readline().split()
        if len(header) < 5 or header[0].lower() != "%%matrixmarket" or header[1].lower() != "matrix":
            raise ValueError(f"{path}: not a Matrix Market matrix file")
        fmt, field, symm = header[2].lower(), header[3].lower(), header[4].lower()
        if fmt != "coordinate":
            raise ValueError(f"{path}: only the coordinate format is read (got {fmt})")
        if field not in ("real", "integer", "pattern", "double"):
            raise ValueError(f"{path}: field {field} is not supported")
        if symm not in ("general", "symmetric", "skew-symmetric"):
            raise ValueError(f"{path}: symmetry {symm} is not supported")
        line = f.readline()
        while line.startswith("%") or not line.strip():
            line = f.readline()
        m, n, nz = (int(t) for t in line.split()[:3])
        ncols = 2 if field == "pattern" else 3
        body = np.loadtxt(f, ndmin=2, max_rows=nz, usecols=range(ncols)) if nz > 0 else np.zeros((0, ncols))
    if body.shape[0] != nz:
        raise ValueError(f"{path}: {body.shape[0]} entries, header says {nz}")
    r = body[:, 0].astype(np.int64) - 1
    c = body[:, 1].astype(np.int64) - 1
    v = np.ones(nz) if field == "pattern" else body[:, 2].astype(np.float64)
    if nz and (r.min() < 0 or c.min() < 0 or r.max() >= m or c.max() >= n):
        raise ValueError(f"{path}: an index lies outside the {m} x {n} matrix")
    if symm != "general":
        off = r != c
        sign = -1.0 if symm == "skew-symmetric" else 1.0
        r, c, v = np.concatenate([r, c[off]]), np.concatenate([c, r[off]]), np.concatenate([v, sign * v[off]])
    order = np.argsort(r, kind="stable")  # rows ascending, file order inside a row
    counts = np.bincount(r, minlength=m)
    ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=ptr[1:])
    if ptr[-1] >= 2**31 or m >= 2**31 or n >= 2**31:
        raise ValueError(f"{path}: too large for 32-bit indices")
    return HostCSR(m, n, ptr.astype(np.int32), c[order].astype(np.int32), v[order], str(path))
