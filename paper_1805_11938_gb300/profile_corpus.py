"""Training data for the format selector, collected on this GPU.

Sec. V-B "Generating Training Data": every training matrix is run in every
representation, repeating until the 95% confidence interval is within 5% of
the mean, the best one is recorded as the label, and the static features are
extracted.  Here the matrices are the seeded synthetic corpus (1000 matrices,
n log-uniform in [1e3, 5e6], five structure families: banded, stencils,
block-diagonal, uniform random, power-law rows) and every step runs in the
library: conversion, spmv_features, and spmv_run timed with CUDA events after
an L2 flush.

Each matrix is timed twice per format:
  * "ms": one product of the matrix alone, the paper's measure (the label of
    the selector used by spmv_select);
  * "ms_batch": the time per copy of a product of the K-fold block-diagonal
    replica diag(A, ..., A) (K copies, about REPLICA_NNZ nonzeros in all; K = 1
    for larger matrices).  That product keeps the whole GPU busy with A's rows,
    as the batched kernel does when it multiplies many matrices at once, so it
    measures a format's throughput on A rather than the latency of a small
    launch (the label of the selector used for batches).

One JSON line per matrix is appended to the output file, so an interrupted run
resumes where it stopped (matrices already in the file are skipped).

--classes 7 times two more candidates beside the five formats, both from
Sec. II/III of the paper and both settings of the library's kernels: plain
SELL (SELL-C-sigma with sigma = 1, no sorting) and the standalone COO format
(HYB with every entry in its COO part, which the library stores grouped by
row).  Such a table names its classes in each line ("classes"); the shipped
selectors keep the five formats.

    python -m paper_1805_11938_gb300.profile_corpus --out table.jsonl [--count 1000] [--classes 7]
    python -m paper_1805_11938_gb300.profile_corpus --refeaturize table.jsonl --out new.jsonl
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FORMAT_CAP_BYTES = 24 << 30  # a padded layout larger than this counts as infeasible (throughput 0)
HYB_K_NONE = -1              # hyb_k: every entry in the COO part (include/spmv.h SPMV_HYB_K_NONE)
# candidate classes: (name, format id, conversion parameters)
CLASSES_5 = [("CSR", 0, {}), ("CSR5", 1, {}), ("ELL", 2, {}), ("SELL", 3, {}), ("HYB", 4, {})]
CLASSES_7 = CLASSES_5 + [("SELL_plain", 3, {"sell_sigma": 1}), ("COO", 4, {"hyb_k": HYB_K_NONE})]
REPLICA_NNZ = 1 << 23        # nonzeros of the block-diagonal replica used for the throughput time


def replica(a, k: int):
    """diag(A, ..., A) with k copies of A (host CSR)."""
    import numpy as np

    import synth

    if k == 1:
        return a
    off = (np.arange(k, dtype=np.int64) * a.nnz)[:, None]
    ptr = np.concatenate([(a.ptr[:-1][None, :].astype(np.int64) + off).ravel(), [k * a.nnz]]).astype(np.int32)
    idx = (a.idx[None, :].astype(np.int64) + (np.arange(k, dtype=np.int64) * a.n)[:, None]).ravel().astype(np.int32)
    val = np.tile(a.val, k)
    return synth.CSR(k * a.m, k * a.n, ptr, idx, val, f"{a.name}_x{k}")


def replica_count(a) -> int:
    if a.nnz == 0 or a.nnz >= REPLICA_NNZ:
        return 1
    k = -(-REPLICA_NNZ // a.nnz)
    return max(1, min(k, (2**31 - 1) // max(a.n, a.m, 1) - 1))


def done_indices(path: str) -> set:
    out = set()
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                try:
                    out.add(json.loads(line)["index"])
                except (ValueError, KeyError):
                    continue
    return out


def _time_formats(a, seed, timer, cap_bytes, measure_kw, classes=CLASSES_5):
    import torch

    import synth
    from . import DeviceCSR, SpmvError, spmv_convert, spmv_run

    d = DeviceCSR.from_host(a)
    x = torch.as_tensor(synth.vector(a.n, seed ^ 0x77)).cuda()
    y = torch.empty(a.m, dtype=torch.float64, device="cuda")
    times, status, conv = {}, {}, {}
    for name, f, params in classes:
        try:
            t0 = time.perf_counter()
            h = spmv_convert(f, d, {"max_bytes": cap_bytes, **params})
            torch.cuda.synchronize()
            conv[name] = 1e3 * (time.perf_counter() - t0)
        except SpmvError as e:
            times[name] = None
            status[name] = e.name
            continue
        r = timer.measure(lambda: spmv_run(h, x, y), **measure_kw)
        times[name] = r["ms"]
        status[name] = f"ci={r['ci_halfwidth_ms'] / r['ms']:.3f} n={r['n']}"
        del h
    return d, times, status, conv


def profile_one(a, spec, timer, cap_bytes: int, measure_kw: dict, classes=CLASSES_5) -> dict:
    from . import spmv_features

    names = [c[0] for c in classes]
    d, times, status, conv = _time_formats(a, spec["seed"], timer, cap_bytes, measure_kw, classes)
    feat = spmv_features(d).cpu().numpy().astype(float).tolist()
    del d
    k = replica_count(a)
    if k == 1:
        times_b = dict(times)
    else:
        _, tb, _, _ = _time_formats(replica(a, k), spec["seed"], timer, cap_bytes, measure_kw, classes)
        times_b = {f: (None if v is None else v / k) for f, v in tb.items()}
    feas = {f: v for f, v in times.items() if v is not None}
    best = min(feas, key=lambda f: feas[f])
    feas_b = {f: v for f, v in times_b.items() if v is not None}
    best_b = min(feas_b, key=lambda f: feas_b[f])
    rec = {"index": spec["index"], "spec": {k2: v for k2, v in spec.items() if k2 != "seed"}, "m": a.m, "nnz": a.nnz,
           "features": feat, "ms": times, "status": status, "convert_ms": conv, "label": names.index(best),
           "best": best, "replicas": k, "ms_batch": times_b, "label_batch": names.index(best_b),
           "best_batch": best_b}
    if classes is not CLASSES_5:
        rec["classes"] = names
    return rec


def run(out: str, count: int = 1000, start: int = 0, cap_bytes: int = FORMAT_CAP_BYTES, n_min: int = 10,
        n_max: int = 60, log=print, classes=CLASSES_5) -> None:
    import synth
    from .autotune import Timer

    have = done_indices(out)
    todo = [i for i in range(start, count) if i not in have]
    timer = Timer()
    kw = {"n_min": n_min, "n_max": n_max, "warmup": 2}
    t_start = time.time()
    with cf.ThreadPoolExecutor(2) as ex, open(out, "a") as fh:
        futs = {}
        for j, i in enumerate(todo[:2]):
            futs[i] = ex.submit(synth.corpus_matrix, i)
        for j, i in enumerate(todo):
            a = futs.pop(i).result()
            if j + 2 < len(todo):
                futs[todo[j + 2]] = ex.submit(synth.corpus_matrix, todo[j + 2])
            rec = profile_one(a, synth.corpus_spec(i), timer, cap_bytes, kw, classes)
            fh.write(json.dumps(rec) + "\n")
            fh.flush()
            if j % 50 == 0:
                log(f"[{j + 1}/{len(todo)}] matrix {i} {rec['spec']['family']} n={a.m} nnz={a.nnz} best={rec['best']} "
                    f"batch best={rec['best_batch']} ({time.time() - t_start:.0f} s)", flush=True)


def refeaturize(table: str, out: str, log=print) -> None:
    """Rewrites a profiled table with the features the library computes now
    (spmv_features on each regenerated matrix); the timings and labels stay."""
    import concurrent.futures as cf2

    import synth
    from . import DeviceCSR, spmv_features

    with open(table) as fh:
        recs = [json.loads(line) for line in fh if line.strip()]
    t0 = time.time()
    with cf2.ThreadPoolExecutor(2) as ex, open(out + ".tmp", "w") as fo:
        futs = {}
        for j, r in enumerate(recs[:2]):
            futs[j] = ex.submit(synth.corpus_matrix, r["index"])
        for j, r in enumerate(recs):
            a = futs.pop(j).result()
            if j + 2 < len(recs):
                futs[j + 2] = ex.submit(synth.corpus_matrix, recs[j + 2]["index"])
            r["features"] = spmv_features(DeviceCSR.from_host(a)).cpu().numpy().astype(float).tolist()
            fo.write(json.dumps(r) + "\n")
            if j % 200 == 0:
                log(f"[{j + 1}/{len(recs)}] ({time.time() - t0:.0f} s)", flush=True)
    os.replace(out + ".tmp", out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--refeaturize", default=None, metavar="TABLE",
                    help="rewrite TABLE's features with the current spmv_features into --out (timings kept)")
    ap.add_argument("--out", required=True)
    ap.add_argument("--count", type=int, default=1000)
    ap.add_argument("--start", type=int, default=0)
    ap.add_argument("--cap-gb", type=float, default=24.0)
    ap.add_argument("--classes", type=int, default=5, choices=(5, 7))
    args = ap.parse_args()
    if args.refeaturize:
        refeaturize(args.refeaturize, args.out)
        return
    run(args.out, args.count, args.start, int(args.cap_gb * (1 << 30)),
        classes=CLASSES_7 if args.classes == 7 else CLASSES_5)


if __name__ == "__main__":
    main()
