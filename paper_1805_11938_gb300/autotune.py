"""Autotuner and profiler for the five formats.

Times spmv_run with CUDA events on the launching stream.  Before every timed
run a buffer larger than L2 is written, so each product starts cold, as it
would between the other kernels of an application.  Repetitions follow the
stopping rule of the paper's training-data collection (Sec. V-B "Generating
Training Data"): repeat until the 95% confidence interval of the mean is
narrower than 5% of the mean, within a minimum and a maximum count.

tune() searches each format's parameters (SELL C and sigma, CSR5 sigma,
the CSR path, HYB K) and keeps the fastest; profile() gives the best time
of every format, the label used to train the selector.
"""
from __future__ import annotations

import math
import statistics

from . import (FORMATS, SPMV_CSR, SPMV_CSR5, SPMV_ELL, SPMV_HYB, SPMV_SELL, SpmvError, spmv_convert,
               spmv_run)

T95 = {2: 12.71, 3: 4.30, 4: 3.18, 5: 2.78, 6: 2.57, 7: 2.45, 8: 2.36, 9: 2.31, 10: 2.26}


def _t95(n: int) -> float:
    return T95.get(n, 1.96 + 2.5 / max(n - 1, 1))


class L2Flush:
    """Evicts L2 between timed runs.  Writes a buffer larger than L2, so that
    nothing a timed kernel touched stays cached, then (clean=True) reads a
    second such buffer, so that the dirty lines of that write are written
    back to memory before the next timed run starts rather than during it
    (where they would add up to L2's size of writes to the kernel's time)."""

    def __init__(self, nbytes: int = 256 << 20, clean: bool = True):
        import torch

        self.w = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.r = torch.zeros(nbytes // 8, dtype=torch.int64, device="cuda") if clean else None
        self.out = torch.zeros((), dtype=torch.int64, device="cuda")
        self.torch = torch

    def __call__(self):
        self.w.zero_()
        if self.r is not None:
            self.torch.sum(self.r, dim=0, out=self.out)

    def describe(self) -> str:
        mib = self.w.numel() >> 20
        return (f"flushed: {mib} MiB written, then {mib} MiB read, before every timed step (the write evicts the "
                f"last step's data, the read writes the flush's dirty lines back before the step)"
                if self.r is not None else f"flushed: {mib} MiB written before every timed step")


class Timer:
    """CUDA-event timing of one callable, L2 flushed (L2Flush) before each run."""

    def __init__(self, flush_bytes: int = 256 << 20):
        import torch

        self.torch = torch
        self.flush = L2Flush(flush_bytes)
        self.stream = torch.cuda.current_stream()

    def once(self, fn) -> float:
        t = self.torch
        s, e = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
        self.flush()
        s.record(self.stream)
        fn()
        e.record(self.stream)
        e.synchronize()
        return s.elapsed_time(e)

    def batch(self, fn, n: int) -> list:
        t = self.torch
        evs = [(t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)) for _ in range(n)]
        for s, e in evs:
            self.flush()
            s.record(self.stream)
            fn()
            e.record(self.stream)
        evs[-1][1].synchronize()
        return [s.elapsed_time(e) for s, e in evs]

    def measure(self, fn, warmup: int = 3, n_min: int = 10, n_max: int = 200, rel_gap: float = 0.05) -> dict:
        """Mean time (ms) with the 95%-CI stopping rule: stop when 2*halfwidth < rel_gap*mean."""
        for _ in range(warmup):
            fn()
        xs = []
        while True:
            xs += self.batch(fn, n_min if not xs else max(5, len(xs) // 2))
            m = statistics.mean(xs)
            sd = statistics.stdev(xs) if len(xs) > 1 else 0.0
            half = _t95(len(xs)) * sd / math.sqrt(len(xs))
            if 2 * half <= rel_gap * m or len(xs) >= n_max:
                return {"ms": m, "ci_halfwidth_ms": half, "n": len(xs), "min_ms": min(xs)}


def default_grid(fmt: int, m: int) -> list:
    if fmt == SPMV_CSR:  # the automatic path choice, the tiles
        return [{}, {"csr_block_nnz": 352}]
    if fmt == SPMV_CSR5:
        return [{"csr5_sigma": s} for s in (8, 12, 16, 24, 32)]
    if fmt == SPMV_ELL:
        return [{}]
    if fmt == SPMV_SELL:
        out = []
        for C in (32, 64, 128):
            for sig in (1, 32 * C, 1024 * C, -1):  # sigma = 1 keeps the rows in place (no perm read)
                if sig == -1 or sig < m:
                    out.append({"sell_C": C, "sell_sigma": sig})
        return out
    return [{"hyb_k": 0}, {"hyb_k": "half"}, {"hyb_k": "double"}]


def tune_format(fmt: int, csr, x, y, timer: Timer, grid=None, max_bytes: int = 0, measure_kw=None) -> dict:
    """Best parameters of one format by exhaustive search over `grid`."""
    grid = grid if grid is not None else default_grid(fmt, csr.m)
    measure_kw = measure_kw or {}
    table, best = [], None
    rule_k = None
    for p in grid:
        p = dict(p)
        if fmt == SPMV_HYB and isinstance(p.get("hyb_k"), str):
            if rule_k is None:
                continue
            p["hyb_k"] = max(1, rule_k // 2) if p["hyb_k"] == "half" else max(1, 2 * rule_k)
        if max_bytes:
            p["max_bytes"] = max_bytes
        try:
            h = spmv_convert(fmt, csr, p)
        except SpmvError as e:
            table.append({"params": p, "status": e.name})
            continue
        info = h.info()
        if fmt == SPMV_HYB and rule_k is None:
            rule_k = info["params"]["hyb_k"]
        r = timer.measure(lambda: spmv_run(h, x, y), **measure_kw)
        r["params"] = {k: v for k, v in info["params"].items() if k != "max_bytes"}
        r["device_bytes"] = info["device_bytes"]
        table.append(r)
        if best is None or r["ms"] < best["ms"]:
            best = r
        del h
    return {"format": FORMATS[fmt], "best": best, "table": table}


def profile(csr, x, y, formats=(0, 1, 2, 3, 4), tuned: bool = False, max_bytes: int = 0, timer: Timer | None = None,
            measure_kw=None) -> dict:
    """Time of every format (default parameters, or tuned), as used for selector labels."""
    timer = timer or Timer()
    out = {}
    for f in formats:
        grid = None if tuned else [{}]
        out[FORMATS[f]] = tune_format(f, csr, x, y, timer, grid=grid, max_bytes=max_bytes, measure_kw=measure_kw)
    return out
