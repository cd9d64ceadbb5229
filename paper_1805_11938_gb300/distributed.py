"""Row-partitioned product over several GPUs, one process per GPU.

One product y = A x shards by rows.  Rank k owns the contiguous rows
[b_k, b_{k+1}), chosen so that every rank holds about nnz / world nonzeros,
keeps all of x (replicated: broadcast once from rank 0) and writes its own
slice of y with its own kernels on its own device buffers.  A single product
needs no other exchange; an iterative method that feeds y back as the next x
gathers the slices every step (all_gather).  The paper's analogue is its
memory-placement study (Sec. IV-A, Fig. 4): every worker multiplies the share
of the matrix held in its own memory.  No rank reads another rank's memory.

The collectives are torch.distributed calls on the process group the caller
initialised (NCCL between GPUs; gloo works the same on CPU tensors).  The
per-rank product is the library (convert once, spmv_run per step) unless a
`multiply(block, x) -> y_block` callable is given.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class HostCSR:
    m: int
    n: int
    ptr: np.ndarray
    idx: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.idx.size)


def row_partition(ptr, parts: int) -> np.ndarray:
    """Boundaries b[0] = 0 <= b[1] <= ... <= b[parts] = M of nnz-balanced row
    blocks: b[k] is the first row whose pointer reaches k * nnz / parts, so a
    block holds nnz / parts nonzeros up to one row.  Without nonzeros the rows
    are split evenly."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    ptr = np.asarray(ptr, dtype=np.int64)
    m = ptr.size - 1
    nnz = int(ptr[-1])
    k = np.arange(parts + 1, dtype=np.int64)
    if nnz == 0:
        b = (k * m) // parts
    else:
        b = np.searchsorted(ptr[:m], (k * nnz + parts - 1) // parts, side="left").astype(np.int64)
        b = np.maximum.accumulate(np.minimum(b, m))
    b[0], b[-1] = 0, m
    return b


def local_csr(a, r0: int, r1: int) -> HostCSR:
    """Rows [r0, r1) of host CSR `a` (all n columns), ptr rebased to 0."""
    p0, p1 = int(a.ptr[r0]), int(a.ptr[r1])
    ptr = (np.asarray(a.ptr[r0:r1 + 1], dtype=np.int64) - p0).astype(np.int32)
    return HostCSR(r1 - r0, a.n, ptr, np.asarray(a.idx[p0:p1], np.int32), np.asarray(a.val[p0:p1], np.float64),
                   f"{getattr(a, 'name', '')}[{r0}:{r1}]")


class RowPartitioned:
    """This rank's row block of A and the exchange steps around its product."""

    def __init__(self, a, rank: int, world: int, dist=None, multiply=None, fmt: int | None = None,
                 params: dict | None = None, model=None, device: str | None = None):
        self.rank, self.world, self.dist = rank, world, dist
        # where this rank's y lives (and, for a rank without rows, the buffer
        # it contributes to the gather): the GPU for the library's product
        self.device = device or ("cuda" if multiply is None else "cpu")
        self.bounds = row_partition(a.ptr, world)
        self.r0, self.r1 = int(self.bounds[rank]), int(self.bounds[rank + 1])
        self.block = local_csr(a, self.r0, self.r1)
        self.n = a.n
        self.multiply = multiply
        self.handle = None
        if multiply is None and self.block.m > 0:
            from . import DeviceCSR, spmv_convert, spmv_select

            d = DeviceCSR.from_host(self.block)
            if fmt is None:
                fmt = spmv_select(d, model) if model is not None else 0
            self.fmt = fmt
            self.handle = spmv_convert(fmt, d, params)
            del d

    @property
    def rows(self) -> int:
        return self.r1 - self.r0

    def broadcast_x(self, x, src: int = 0):
        """x replicated on every rank (in place)."""
        if self.dist is not None and self.world > 1:
            self.dist.broadcast(x, src)
        return x

    def run(self, x, y_block=None, stream=None):
        """y_block = (rows r0..r1 of A) x, on this rank."""
        if self.multiply is not None:
            return self.multiply(self.block, x)
        from . import spmv_run

        if self.block.m == 0:
            return y_block if y_block is not None else x.new_empty(0)
        return spmv_run(self.handle, x, y_block, stream)

    def gather_y(self, y_block):
        """The whole y on every rank: the blocks in row order (all_gather of
        blocks padded to the longest)."""
        import torch

        if self.dist is None or self.world == 1:
            return y_block
        sizes = np.diff(self.bounds)
        width = int(sizes.max())
        buf = torch.zeros(width, dtype=torch.float64, device=y_block.device if y_block is not None else self.device)
        if self.rows:
            buf[:self.rows] = y_block
        parts = [torch.empty_like(buf) for _ in range(self.world)]
        self.dist.all_gather(parts, buf)
        return torch.cat([p[:int(s)] for p, s in zip(parts, sizes)])
