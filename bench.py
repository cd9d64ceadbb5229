#!/usr/bin/env python
"""Benchmark: FP64 SpMV on the GB300 through the library's C ABI.

One step = the deployment path on one matrix resident in HBM: the selector
kernel (features + scaling + network, result kept on the device) and the
product y = A x in the format the selector chose for this matrix.  The
step's two kernels are captured once as a CUDA graph that every timed step
replays (--no-graph launches them directly).  Every format is also timed on
its own; conversions are timed once.  Between timed steps a 256 MiB buffer is
written to flush L2, and each step is bracketed by CUDA events on the stream
the kernels run on.  Every row of the timed result is checked against the
oracle.

The default workload is the largest single-GPU one, the 27-point stencil on
224^3 (300.8 M nonzeros); the 2e6-row power-law matrix and the 2e7-row
power-law graph are then measured the same way with fewer steps and carried
in the same line under "extra_workloads".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...     # the CPU oracle on the host cores

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1805_11938_gb300.autotune import L2Flush  # noqa: E402

METRIC = "FP64 SpMV GFLOP/s & HBM GB/s vs ~8 TB/s; selector % of best-format throughput"
FORMATS = ("CSR", "CSR5", "ELL", "SELL", "HYB")

WORKLOADS = {
    "powerlaw_2e6": "n = 2,000,000, row lengths ceil(Pareto alpha 2.1) on [1, 5000], uniform columns, N(0,1) values",
    "laplacian_64": "2D 5-point Laplacian on 64 x 64 (n = 4096, nnz = 20224)",
    "stencil27_224": "3D 27-point stencil on 224^3 (n = 11,239,424, nnz = 300,763,000)",
    "graph_2e7": "n = 20,000,000 power-law graph, mean about 12 entries per row, at most 1e5",
    "batch512": "512 matrices, rows log-uniform in [1e3, 2e5], row lengths in [3, 200] (half uniform, half "
                "power-law), one persistent launch replayed from a CUDA graph",
    # scaled-down cases of the two large configurations, for hardware-counter
    # captures (inputs larger than L2, a few GB on the device)
    "stencil27_112": "3D 27-point stencil on 112^3 (n = 1,404,928, nnz = 37,259,704): the 224^3 stencil scaled down",
    "graph_1e7_lite": "1e7 rows x 2e7 columns (x 160 MB, as the 2e7 graph's), row lengths ceil(Pareto alpha 2.1) "
                      "on [1, 1e5], uniform columns: the 2e7 graph scaled down",
}


def make_matrix(name: str):
    import synth

    if name == "powerlaw_2e6":
        return synth.config2()
    if name == "laplacian_64":
        return synth.config1()
    if name == "stencil27_224":
        return synth.config5_stencil()
    if name == "graph_2e7":
        return synth.config5_graph()
    if name == "stencil27_112":
        return synth.config5_stencil(112)
    if name == "graph_1e7_lite":
        lens = synth.powerlaw_lengths(10_000_000, synth.seed_of(5, 2), xmax=1e5, lmax=100_000)
        return synth.from_lengths_random_cols(lens, 20_000_000, synth.seed_of(5, 2), "graph_1e7_lite")
    raise SystemExit(f"unknown workload {name}")


def dist_backend() -> tuple:
    """The process group's backend and the device its tensors live on: NCCL
    between GPUs; SPMV_BENCH_BACKEND=gloo runs the same ranks' exchanges on the
    host (for checking the multi-rank path where only one GPU is at hand --
    the ranks' kernels never wait on one another)."""
    b = os.environ.get("SPMV_BENCH_BACKEND", "nccl")
    return b, ("cuda" if b == "nccl" else "cpu")


def reduce_over_ranks(total_ms: float, flops: float, dist=None, device: str = "cpu") -> tuple:
    """Whole-job rate over the ranks: the slowest rank's timed total (max) and
    every rank's flops (sum); returns (max total ms, GFLOP/s).  Each rank
    multiplies its own row block of the one matrix (x broadcast once at setup)
    or its own share of a batch, so the timed steps exchange nothing else."""
    if dist is not None:
        import torch

        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        f = torch.tensor([float(flops)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
        total_ms, flops = float(t.item()), float(f.item())
    return total_ms, flops / (total_ms * 1e6)


def algorithmic_bytes(fmt: int, info: dict) -> int:
    """Bytes a format must move per product: every stored nonzero once (8 B value + 4 B index),
    x and y once, plus the format's per-row / per-unit metadata (never the padding)."""
    m, n, nnz = info["m"], info["n"], info["nnz"]
    base = 12 * nnz + 8 * n + 8 * m
    aux = info["aux"]
    if fmt == 0:  # CSR: row pointers
        return base + 4 * (m + 1)
    if fmt == 1:  # CSR5: per tile 32 flag words, tile_ptr, empty_ptr, the head row's pointer, join slots
        return base + aux[0] * (128 + 4 + 8 + 4 + 16)
    if fmt == 2:  # ELL: row_len
        return base + 4 * m
    if fmt == 3:  # SELL: row_len, perm (not read when the sort moved no row: aux[3] = -1), slice_ptr, units
        return base + (4 if aux[3] == -1 else 8) * m + 8 * (aux[0] + 1) + 8 * aux[1]
    # HYB: ELL row_len + tail row ids and pointers + read-modify-write of tail rows' y
    return base + 4 * m + 8 * aux[1] + 8 * aux[1]


# kernels of one selection (include/spmv.h, spmv_select_async): the exact pass
# over ptr and the features cluster
SELECT_LAUNCHES = 2


def launches_per_run(fmt: int, info: dict) -> int:
    """Kernels one spmv_run launches (include/spmv.h, spmv_run)."""
    aux = info["aux"]
    if fmt == 1:
        return 1 if (aux[0] > 0 or aux[2] > 0) else 0
    if fmt == 3:  # one launch per column panel and one putting y back in row order
        return aux[3] + 1 if aux[3] > 0 else 1
    if fmt == 4:
        return 1 + (1 if aux[1] > 0 else 0)
    return 1


def batch_families(infos) -> set:
    """Task families of a batch (include/spmv.h, spmv_batch_build): one
    persistent kernel per family present runs in each replay.  CSR5, ELL, the
    ELL part of HYB, CSR on the lanes-per-row path and CSR without nonzeros
    share one family; SELL has one per chunk size C = 32, 64, 128; CSR tiles
    and HYB tails have their own."""
    families = set()
    for i in infos:
        f, aux = i["fmt"], i["aux"]
        if f == 0:
            families.add("csr" if aux[0] > 0 and aux[1] == 0 else "other")
        elif f == 3:
            if aux[1] > 0:
                families.add({32: "sell32", 64: "sell64"}.get(i["params"]["sell_C"], "sell128"))
        else:
            families.add("other")
            if f == 4 and aux[1] > 0:
                families.add("hyb_tail")
    return families


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self) -> dict:
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rate(a, x, seconds: float) -> dict:
    """The oracle as it stands on the host: its rows split over every core the
    process may use (the threaded loop gives the single-threaded result bit
    for bit), and the single-threaded loop beside it; half the time each."""
    import oracle

    cores = host_cores()

    def rate(fn, budget):
        fn()  # warm
        reps, t0 = 0, time.perf_counter()
        while True:
            fn()
            reps += 1
            el = time.perf_counter() - t0
            if el >= budget:
                return reps, el

    r1, e1 = rate(lambda: oracle.csr_spmv(a, x), seconds / 2)
    rn, en = rate(lambda: oracle.csr_spmv_threads(a, x, cores), seconds / 2)
    return {"value": 2.0 * a.nnz * rn / en / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{rn} full products of the {a.m}-row matrix ({a.nnz} nonzeros), C, rows split over {cores} "
                      f"threads, {en:.1f} s",
            "single_core": {"value": 2.0 * a.nnz * r1 / e1 / 1e9, "cores": 1,
                            "sample": f"{r1} full products, single-threaded C, {e1:.1f} s"}}


REF_BLOCK_NNZ = 1 << 22


def row_blocks(a, block_nnz: int):
    """Contiguous row blocks of about block_nnz nonzeros each (views, not copies)."""
    import synth

    out, r0 = [], 0
    while r0 < a.m:
        r1 = int(np.searchsorted(a.ptr, a.ptr[r0] + block_nnz, side="right")) - 1
        r1 = min(max(r1, r0 + 1), a.m)
        p0 = int(a.ptr[r0])
        out.append(synth.CSR(r1 - r0, a.n, (a.ptr[r0:r1 + 1] - p0).astype(np.int32), a.idx[p0:a.ptr[r1]],
                             a.val[p0:a.ptr[r1]], f"rows{r0}"))
        r0 = r1
    return out


def run_reference(args, rank: int, world: int) -> None:
    """The CPU oracle as it stands on the host cores; one step = the product of
    one row block of about 2^22 nonzeros, cycling over the whole matrix, its
    rows split over every core the process may use."""
    if rank != 0:
        return
    import synth
    import oracle

    a = make_matrix(args.workload)
    x = synth.vector(a.n, 1)
    blocks = row_blocks(a, REF_BLOCK_NNZ)
    cores = host_cores()
    for i in range(args.warmup):
        oracle.csr_spmv_threads(blocks[i % len(blocks)], x, cores)
    flops, t = 0, 0.0
    for i in range(args.steps):
        b = blocks[i % len(blocks)]
        t0 = time.perf_counter()
        oracle.csr_spmv_threads(b, x, cores)
        t += time.perf_counter() - t0
        flops += 2 * b.nnz
    v = flops / t / 1e9
    sample = (f"{args.steps} row blocks of about {REF_BLOCK_NNZ} nonzeros ({flops // 2} nonzeros in all) of the "
              f"{a.m}-row matrix, C, rows split over {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak" if args.workload == "batch512" else "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "n": a.m, "nnz": a.nnz,
                       "step": "CPU oracle product of one row block (about 2^22 nonzeros)"},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


TUNE_MARGIN = 0.03  # batch tuning: how much faster a later grid entry must be to replace an earlier one


def tuning_grid(fmt: int) -> list:
    """The autotuner's small per-format grid (the batched workload tunes every
    matrix with it; the single-matrix workloads tune the selected format)."""
    if fmt == 1:
        return [{"csr5_sigma": 16}, {"csr5_sigma": 24}, {"csr5_sigma": 32}]
    if fmt == 3:
        return [{"sell_C": 32, "sell_sigma": -1}, {"sell_C": 64, "sell_sigma": -1}, {"sell_C": 32, "sell_sigma": 1024},
                {"sell_C": 64, "sell_sigma": 1}, {"sell_C": 128, "sell_sigma": -1}]
    if fmt == 0:  # the automatic path choice and the tiles
        return [{}, {"csr_block_nnz": 352}]
    return [{}]


class BatchWorkload:
    """n_mat matrices of the batched configuration, each in the format the
    batch selector picks (parameters from the autotuner's grid when tune),
    multiplied by the persistent launches replayed from a CUDA graph: the
    kernels per task family, and one launch for every task
    (SPMV_BATCH_ONE_LAUNCH); both against the same products as n_mat separate
    launches (also a graph)."""

    def __init__(self, n_mat, args, rank, tune=True, mixed=False):
        import torch

        import synth
        import paper_1805_11938_gb300 as sp
        from paper_1805_11938_gb300 import autotune

        self.torch, self.sp = torch, sp
        self.model_path = sp.MODEL_BATCH_PATH if os.path.exists(sp.MODEL_BATCH_PATH) else sp.MODEL_PATH
        model = sp.Model.load(self.model_path)
        timer = autotune.Timer()
        self.handles, self.xs, self.ys, self.infos, self.mats = [], [], [], [], []
        self.counts = [0] * 5
        self.params_mix = {}
        t0 = time.perf_counter()
        for j in range(n_mat):
            a = synth.batch_matrix(j + rank * n_mat)
            d = sp.DeviceCSR.from_host(a)
            if mixed:  # every format in turn
                f = j % 5
            else:
                f = sp.spmv_select(d, model) if args.batch_format < 0 else args.batch_format
            x = torch.as_tensor(synth.vector(a.n, 900 + j)).cuda()
            y = torch.empty(a.m, dtype=torch.float64, device="cuda")
            best = None
            for p in (tuning_grid(f) if tune else [{}]):
                h = sp.spmv_convert(f, d, p)
                ms = timer.measure(lambda: sp.spmv_run(h, x, y), warmup=1, n_min=5, n_max=10)["ms"] if tune else 0.0
                # a later grid entry must win by TUNE_MARGIN: near-ties keep the earlier entry, so
                # timing noise does not change the batch's parameter mix from run to run
                if best is None or ms < best[0] * (1.0 - TUNE_MARGIN):
                    best = (ms, h, p)
            self.handles.append(best[1])
            self.infos.append(best[1].info())
            key = ",".join(f"{k}={v}" for k, v in sorted(best[2].items())) or "default"
            self.params_mix[key] = self.params_mix.get(key, 0) + 1
            self.xs.append(x)
            self.ys.append(y)
            self.counts[f] += 1
            if j < 8:
                self.mats.append((a, j))
            del d
        self.setup_s = time.perf_counter() - t0
        self.total_nnz = sum(i["nnz"] for i in self.infos)
        self.total_rows = sum(i["m"] for i in self.infos)
        self.b = sp.Batch(self.handles)
        self.b1 = sp.Batch(self.handles, one_launch=True)
        self.flush = L2Flush()
        self.stream = torch.cuda.current_stream()

    def timed(self, fn, n, warm):
        torch, flush, stream = self.torch, self.flush, self.stream
        for _ in range(warm):
            flush()
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for s0, e0 in evs:
            flush()
            s0.record(stream)
            fn()
            e0.record(stream)
        torch.cuda.synchronize()
        return [s0.elapsed_time(e0) for s0, e0 in evs]

    def compare(self, steps, warmup) -> dict:
        """Times the three ways; y of each equals the separate products bit for bit."""
        torch = self.torch
        ys1 = [torch.empty_like(y) for y in self.ys]
        ys2 = [torch.empty_like(y) for y in self.ys]
        t_one = self.timed(lambda: self.b1.run(self.xs, ys1), steps, warmup)
        t_sep = self.timed(lambda: self.b.run_separate(self.xs, ys2), steps, warmup)
        t_fam = self.timed(lambda: self.b.run(self.xs, self.ys), steps, warmup)
        same = all(torch.equal(u, v) and torch.equal(u, w) for u, v, w in zip(self.ys, ys1, ys2))
        ab = sum(algorithmic_bytes(i["fmt"], i) for i in self.infos)
        tf, t1, ts = statistics.mean(t_fam), statistics.mean(t_one), statistics.mean(t_sep)
        return {"matrices": len(self.handles), "rows": self.total_rows, "nnz": self.total_nnz,
                "formats": dict(zip(FORMATS, self.counts)), "format_choice": os.path.basename(self.model_path),
                "params_mix": self.params_mix, "family_kernels_ms": tf, "family_launches": self.b.launches(),
                "one_launch_ms": t1, "one_launch_launches": self.b1.launches(), "separate_ms": ts,
                "speedup_families_over_separate": ts / tf, "speedup_one_launch_over_separate": ts / t1,
                "faster": "family kernels" if tf <= t1 else "one launch",
                "gflops_families": 2.0 * self.total_nnz / tf / 1e6, "gflops_one_launch": 2.0 * self.total_nnz / t1 / 1e6,
                "alg_bytes": ab, "alg_gbs_best": ab / min(tf, t1) / 1e6, "bitwise_equal_all_three": same,
                "setup_s": self.setup_s, "t_fam": t_fam, "t_one": t_one}

    def check(self) -> bool:
        import oracle

        oks = []
        for a, j in self.mats:
            yv = self.ys[j].cpu().numpy()
            xv = self.xs[j].cpu().numpy()
            oks.append(bool(np.all(np.abs(yv - oracle.csr_spmv(a, xv)) <= oracle.fp_bound(a, xv))))
        return all(oks)


def run_batch(args, rank: int, world: int) -> None:
    """The batched configuration: each rank multiplies its own share of
    batch_count matrices (weak scaling).  The headline is the faster of the
    two persistent ways, per replay."""
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0")) % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(dist_backend()[0])
    import paper_1805_11938_gb300 as sp

    sp.lib()
    bw = BatchWorkload(args.batch_count, args, rank)
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        cmp = bw.compare(args.steps, args.warmup)
    clocks = clk.summary()
    t_fam, t_one = cmp.pop("t_fam"), cmp.pop("t_one")
    t_b = t_fam if cmp["faster"] == "family kernels" else t_one  # the headline: the faster way
    tb = statistics.mean(t_b)
    total_b, value = reduce_over_ranks(sum(t_b), 2.0 * bw.total_nnz * args.steps, dist, dist_backend()[1])
    launches_per_replay = bw.b.launches() if cmp["faster"] == "family kernels" else bw.b1.launches()
    peak, src = load_peaks()
    batch_traffic = None
    if args.batch_format < 0:
        batch_traffic = load_traffic(f"batch{args.batch_count}:{os.path.basename(bw.model_path)}")
    families = batch_families(bw.infos)
    ab = cmp["alg_bytes"]
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_b / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch512", "description": WORKLOADS["batch512"], "matrices": args.batch_count,
                       "rows": bw.total_rows, "nnz": bw.total_nnz, "formats": dict(zip(FORMATS, bw.counts)),
                       "format_choice": (os.path.basename(bw.model_path) if args.batch_format < 0 else "fixed"),
                       "l2": bw.flush.describe(), "setup_s": bw.setup_s,
                       "step": f"one graph replay of the persistent batched launches ({cmp['faster']})"},
            "roofline": {"bound": "hbm", "achieved": ab / tb / 1e6, "peak": peak, "unit": "GB/s",
                         "frac": ab / tb / 1e6 / peak, "traffic": batch_traffic,
                         "kernel": f"persistent batched product ({launches_per_replay} kernels per replay; family "
                                   f"kernels present: {', '.join(sorted(families))}); traffic summed over them",
                         "alg_bytes_per_launch": ab, "peak_source": f"{src} hbm_gbs"},
            "batch": cmp, "gpu_launches": world * args.steps * launches_per_replay, "clocks": clocks}
    if rank == 0 and not args.no_cpu_baseline:
        line["check"] = {"first_8_matrices_within_bound": bw.check()}
        a0, j0 = bw.mats[0]
        line["cpu_baseline"] = cpu_oracle_rate(a0, bw.xs[j0].cpu().numpy(), min(args.cpu_seconds, 5.0))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def load_peaks() -> tuple:
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = {}
    if os.path.exists(pk):
        with open(pk) as fh:
            peaks = json.load(fh)
    peak = peaks.get("hbm_gbs")
    return (peak, "measured") if peak else (6800.0, "fallback")


def load_traffic(key: str, params: dict | None = None):
    """DRAM bytes per launch from an ncu capture (profiles/traffic.json).  An
    entry recorded with the tuning parameters of the captured launch counts
    only for a handle with the same resolved parameters; otherwise null."""
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tr_path):
        return None
    with open(tr_path) as fh:
        v = json.load(fh).get(key)
    if not isinstance(v, (dict, list)):
        return v
    for e in v if isinstance(v, list) else [v]:
        want = e.get("params", {})
        if params is not None and all(params.get(k) == w for k, w in want.items()):
            return e["bytes"]
    return None


class Workload:
    """One matrix resident in HBM, measured the way the headline step runs:
    every format converted and timed on its own (the exhaustive search, also
    the yardstick of the selector), the selector's pick and its autotuned parameters,
    the step (selector kernel + product, one CUDA graph) timed with the L2
    flushed before every step, the product kernel's own duration, the gather
    ceiling of the matrix's index stream, and every row of the result checked
    against the oracle."""

    def __init__(self, name, args, sp, torch, stream, flush, model, format_steps, rank=0, world=1, dist=None):
        import synth

        self.name, self.sp, self.torch, self.stream, self.flush = name, sp, torch, stream, flush
        self.fixed_params = args.params if name == args.workload else None
        full = make_matrix(name)
        self.total_nnz, self.total_rows = full.nnz, full.m
        if world > 1:
            # this rank's nnz-balanced row block of the one product (x replicated)
            from paper_1805_11938_gb300.distributed import local_csr, row_partition

            b = row_partition(full.ptr, world)
            self.rows = (int(b[rank]), int(b[rank + 1]))
            full = local_csr(full, *self.rows)
        else:
            self.rows = (0, full.m)
        self.a = a = full
        self.xh = synth.vector(a.n, 1)
        self.d = sp.DeviceCSR.from_host(a)
        self.x = torch.as_tensor(self.xh).cuda()
        if dist is not None:  # x replicated from rank 0 (the one exchange of a single product)
            if dist_backend()[1] == "cuda":
                dist.broadcast(self.x, 0)
            else:
                xc = self.x.cpu()
                dist.broadcast(xc, 0)
                self.x.copy_(xc)
        self.y = torch.empty(a.m, dtype=torch.float64, device="cuda")
        self.model = model
        self.format_steps = format_steps
        self.args = args

    def timed(self, fn, n, warm):
        torch, flush, stream = self.torch, self.flush, self.stream
        for _ in range(warm):
            flush()
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for s, e in evs:
            flush()
            s.record(stream)
            fn()
            e.record(stream)
        torch.cuda.synchronize()
        return [s.elapsed_time(e) for s, e in evs]

    def setup(self):
        """Conversions, per-format times, selection, gather ceiling, tuning."""
        sp, torch, a, d, x, y, args = self.sp, self.torch, self.a, self.d, self.x, self.y, self.args
        # Each format is converted twice: the first call also pays one-time
        # costs (loading the kernels on first launch), the second is the steady
        # cost ("conversion_ms"; the first in "conversion_first_ms").
        fmts = [int(f) for f in args.formats.split(",") if f != ""]
        handles, infos, conv_ms, conv_first_ms, status = {}, {}, {}, {}, {}
        for f in fmts:
            params = {"max_bytes": int(args.ell_cap_gb * (1 << 30))} if f == 2 else None
            h = None
            try:
                for rep in range(2):
                    h = None
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    h = sp.spmv_convert(f, d, params)
                    torch.cuda.synchronize()
                    (conv_first_ms if rep == 0 else conv_ms)[FORMATS[f]] = 1e3 * (time.perf_counter() - t0)
            except sp.SpmvError as e:
                status[FORMATS[f]] = e.name
                continue
            handles[f], infos[f] = h, h.info()
        per_fmt = {}
        for f, h in handles.items():
            ms = statistics.mean(self.timed(lambda h=h: sp.spmv_run(h, x, y), self.format_steps, 5))
            ab = algorithmic_bytes(f, infos[f])
            per_fmt[FORMATS[f]] = {"ms": ms, "gflops": 2 * a.nnz / ms / 1e6, "alg_gbs": ab / ms / 1e6,
                                   "alg_bytes": ab, "device_bytes": infos[f]["device_bytes"],
                                   "params": {k: v for k, v in infos[f]["params"].items() if k != "max_bytes"}}
        for name, st in status.items():
            per_fmt[name] = {"status": st}
        best = min((f for f in handles), key=lambda f: per_fmt[FORMATS[f]]["ms"])

        # ---- selector: the network's own pick; should it name a format whose
        # conversion failed here, the step runs the exhaustive best instead and
        # the line says so (the pick still scores 0 % of best, as an infeasible
        # format does in the corpus evaluation)
        self.fmt_dev = torch.zeros(1, dtype=torch.int32, device="cuda")
        feat = torch.empty(16, dtype=torch.float32, device="cuda")
        model = self.model
        if model is not None:
            pick = sp.spmv_select(d, model)
            fell_back = pick not in handles
            chosen = best if fell_back else pick
            self.select_step = lambda: sp.spmv_select_async(d, model, self.fmt_dev)  # noqa: E731
            kind = "mlp"
        else:
            pick, fell_back, chosen = best, False, best
            self.select_step = lambda: sp.spmv_features(d, feat)  # noqa: E731
            kind = "exhaustive (no trained model found; the step runs the features kernel)"
        sel_ms = statistics.mean(self.timed(self.select_step, self.format_steps, 5))
        pick_ms = per_fmt.get(FORMATS[pick], {}).get("ms")
        self.selector = {"kind": kind, "pick": FORMATS[pick], "chosen": FORMATS[chosen], "best": FORMATS[best],
                         "fell_back": fell_back,
                         "pct_of_best": (100.0 * per_fmt[FORMATS[best]]["ms"] / pick_ms) if pick_ms else 0.0,
                         "select_us": 1e3 * sel_ms, "select_frac_of_spmv": sel_ms / per_fmt[FORMATS[chosen]]["ms"]}

        # ---- gather ceiling of this matrix's index stream: val[k] * x[idx[k]]
        # for every entry, one gather and one DFMA each, no row structure
        from paper_1805_11938_gb300 import probe

        probe_part = torch.empty(probe.partials(), dtype=torch.float64, device="cuda")
        self.probe_ms = statistics.mean(self.timed(lambda: probe.gather(d, x, probe_part), self.format_steps, 5))

        # ---- the selected format's parameters from the autotuner's grid
        # (one-off setup, like the conversion): the fastest of the default and the grid
        hc = handles[chosen]
        fixed = json.loads(self.fixed_params) if self.fixed_params else None
        if fixed is not None:  # --params: these parameters, no search (profiling the kernel a run picked)
            hc = sp.spmv_convert(chosen, d, fixed)
        tune_runs = max(10, min(self.format_steps, 50))
        tune_ms = statistics.mean(self.timed(lambda: sp.spmv_run(hc, x, y), tune_runs, 3))
        tuning = [{"params": fixed if fixed is not None else "default", "ms": tune_ms}]
        for p in tuning_grid(chosen) if fixed is None else []:
            if not p:
                continue
            try:
                h2 = sp.spmv_convert(chosen, d, p)
            except sp.SpmvError as e:
                tuning.append({"params": p, "status": e.name})
                continue
            t2 = statistics.mean(self.timed(lambda h2=h2: sp.spmv_run(h2, x, y), tune_runs, 3))
            tuning.append({"params": p, "ms": t2})
            if t2 < tune_ms:
                hc, tune_ms = h2, t2
            del h2
        # only the tuned handle stays resident (the 119 GB ELL of the power-law
        # matrix, for one, is released here)
        del handles
        torch.cuda.empty_cache()
        self.hc, self.chosen, self.best = hc, chosen, best
        self.info_c = hc.info()
        self.per_fmt, self.tuning = per_fmt, tuning
        self.conv_ms, self.conv_first_ms = conv_ms, conv_first_ms

    def step(self):
        self.select_step()
        self.sp.spmv_run(self.hc, self.x, self.y)

    def capture(self, warmup, use_graph=True):
        """Warm-up, then the step's two launches captured once as a CUDA graph."""
        torch = self.torch
        for _ in range(warmup):
            self.flush()
            self.step()
        torch.cuda.synchronize()
        self.graph = None
        if use_graph:
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self.step()
            torch.cuda.synchronize()
            for _ in range(warmup):
                self.flush()
                self.graph.replay()
        return self.graph.replay if self.graph is not None else self.step

    def kernel_pass(self, n):
        """The product kernel's own duration for the roofline: the steps once
        more, launched directly with an event between the two kernels (an event
        there delays the second launch by a few microseconds, so it stays out
        of the headline loop)."""
        torch, stream = self.torch, self.stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for s, mid, e in ev:
            self.flush()
            s.record(stream)
            self.select_step()
            mid.record(stream)
            self.sp.spmv_run(self.hc, self.x, self.y)
            e.record(stream)
        torch.cuda.synchronize()
        return [m.elapsed_time(e) for _, m, e in ev], statistics.mean(s.elapsed_time(e) for s, _, e in ev)

    def roofline(self, kms):
        peak, src = load_peaks()
        ab = algorithmic_bytes(self.chosen, self.info_c)
        achieved = ab / kms / 1e6
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": load_traffic(f"{self.name}:{FORMATS[self.chosen]}", self.info_c["params"]),
                "kernel": f"{FORMATS[self.chosen]} product", "kernel_ms": kms,
                "kernel_ms_source": "CUDA events around the product in a second pass of the same steps",
                "alg_bytes_per_launch": ab, "peak_source": f"{src} hbm_gbs (STREAM-style copy, burst)",
                "gather_ceiling": {"ms": self.probe_ms, "g_gathers_per_s": self.a.nnz / self.probe_ms / 1e6,
                                   "frac": self.probe_ms / kms,
                                   "what": "the gather probe on this matrix's idx/val: one random gather and one "
                                           "DFMA per entry, no row structure, L2 flushed; frac = its time / the "
                                           "product's"}}

    def check_all_rows(self):
        """Every row of the timed steps' y against the oracle, within the FP64 bound."""
        import oracle

        yv = self.y.cpu().numpy()
        ref = oracle.csr_spmv_threads(self.a, self.xh, host_cores())
        bound = oracle.fp_bound(self.a, self.xh)
        bad = ~(np.abs(yv - ref) <= bound)
        return {"rows": int(self.a.m), "rows_outside_bound": int(bad.sum()), "all_within_bound": not bool(bad.any()),
                "against": "oracle (CPU, rows split over the host cores)"}

    def summary(self, step_ms, kms):
        tuned = {k: v for k, v in self.info_c["params"].items() if k != "max_bytes"}
        return {"description": WORKLOADS[self.name], "n": self.a.m, "nnz": self.a.nnz,
                "selected_format": FORMATS[self.chosen], "exhaustive_best": FORMATS[self.best],
                "selected_params": tuned, "step_ms": step_ms, "gflops": 2.0 * self.a.nnz / step_ms / 1e6,
                "roofline": self.roofline(kms), "formats": self.per_fmt, "selector": self.selector,
                "tuning": self.tuning, "conversion_ms": self.conv_ms}


def measure_extra(name, args, sp, torch, stream, flush, model) -> dict:
    """A further workload on the same GPU, after the headline: the same
    measurements with fewer steps (carried in the JSON line as an extra key)."""
    w = Workload(name, args, sp, torch, stream, flush, model, max(20, min(args.format_steps, 100)))
    w.setup()
    run_step = w.capture(3)
    n = max(20, min(args.steps, 300))
    step_ms = statistics.mean(w.timed(run_step, n, 3))
    kern, _ = w.kernel_pass(n)
    out = w.summary(step_ms, statistics.mean(kern))
    out["steps"] = n
    out["check"] = w.check_all_rows()
    del w
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="stencil27_224", choices=sorted(WORKLOADS))
    ap.add_argument("--extras", default=None,
                    help="comma-separated further workloads measured after the headline and reported as extra keys "
                         "(default: powerlaw_2e6,graph_2e7 beside the stencil; '' for none)")
    ap.add_argument("--ell-cap-gb", type=float, default=160.0, help="ELL footprint cap (the 2e6 power-law ELL is ~119 GB)")
    ap.add_argument("--format-steps", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--formats", default="0,1,2,3,4")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-extra", type=int, default=32,
                    help="after the headline: the first N matrices of the batched configuration as an extra key (0: none)")
    ap.add_argument("--batch-format", type=int, default=-1, help="batch512: one format for every matrix (-1: selector)")
    ap.add_argument("--params", default=None,
                    help="JSON tuning parameters of the headline workload's selected format, used as given "
                         "instead of the autotuner's search (for profiling one kernel)")
    ap.add_argument("--no-graph", action="store_true", help="launch the timed steps directly instead of replaying a CUDA graph")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch512":
        run_batch(args, rank, world)
        return
    if args.extras is None:
        args.extras = "powerlaw_2e6,graph_2e7" if args.workload == "stencil27_224" else ""
    extras = [e for e in args.extras.split(",") if e]
    for e in extras:
        if e not in WORKLOADS or e == "batch512":
            raise SystemExit(f"unknown extra workload {e}")

    import torch

    local = int(os.environ.get("LOCAL_RANK", "0")) % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(dist_backend()[0])

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    import paper_1805_11938_gb300 as sp

    sp.lib()
    flush = L2Flush()
    stream = torch.cuda.current_stream()
    model = sp.Model.load(sp.MODEL_PATH) if os.path.exists(sp.MODEL_PATH) else None

    w = Workload(args.workload, args, sp, torch, stream, flush, model, args.format_steps, rank, world, dist)
    w.setup()
    a, x, y, xh = w.a, w.x, w.y, w.xh

    # ---- timed steps (the headline).  The step's two launches (the selector
    # kernel, the product) are captured once as a CUDA graph and the graph is
    # replayed every step: each replay runs both kernels in full, without the
    # host between them.
    run_step = w.capture(args.warmup, not args.no_graph)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        t_wall = time.perf_counter()
        for s, e in ev:
            flush()
            s.record(stream)
            run_step()
            e.record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_ms, value = reduce_over_ranks(sum(step_ms), 2.0 * a.nnz * args.steps, dist, dist_backend()[1])
    clocks = clk.summary()
    kern_ms, eager_step_ms = w.kernel_pass(args.steps)
    check = w.check_all_rows() if rank == 0 else None
    # the same steps after a write-only flush (its dirty lines then go back to
    # memory during the step), for comparison with the headline's flush
    dirty = L2Flush(clean=False)
    w.flush = dirty
    dirty_ms = statistics.mean(w.timed(run_step, max(20, min(args.steps, 200)), 3))
    w.flush = flush
    del dirty

    # ---- end to end through the library's host-memory call (spmv_run_host):
    # every step copies its x in from pinned host memory, runs the step, and
    # copies its y out.  The io alternates between two device staging pairs
    # and copies on two streams of its own (in and out), so one step's copies
    # overlap the neighbouring steps' compute; every step still moves its own
    # 16 bytes per row.  The working set (the matrix) exceeds L2, so no flush
    # between steps.
    n_e2e = max(10, min(args.steps, 500))
    xh_pin = [torch.as_tensor(xh).pin_memory() for _ in range(2)]
    yh_pin = [torch.empty(a.m, dtype=torch.float64).pin_memory() for _ in range(2)]
    io = sp.HostIO(w.hc)

    def e2e_run(n):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t1.record(stream)  # created now; recorded again after the last copy out
        torch.cuda.synchronize()
        t0.record(stream)
        for i in range(n):
            b = i % 2
            w.select_step()
            io.run(xh_pin[b], yh_pin[b], stream, done=t1 if i == n - 1 else None)
        t1.synchronize()
        return t0.elapsed_time(t1) / n

    e2e_run(5)
    e2e_windows = []
    for _ in range(3):  # the copies cross host memory that other processes share: median of three windows
        barrier()
        e2e_windows.append(e2e_run(n_e2e))
    e2e_ms = statistics.median(e2e_windows)
    torch.cuda.synchronize()
    e2e_ms, e2e_value = reduce_over_ranks(e2e_ms, 2.0 * a.nnz, dist, dist_backend()[1])
    e2e_same = bool(np.array_equal(yh_pin[(n_e2e - 1) % 2].numpy(), y.cpu().numpy()))
    agree = None
    if model is not None:
        torch.cuda.synchronize()
        agree = FORMATS[int(w.fmt_dev.item())] == w.selector["pick"]
    del io, xh_pin, yh_pin

    kms = statistics.mean(kern_ms)
    summ = w.summary(total_ms / args.steps, kms)
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "n": a.n, "nnz": w.total_nnz,
                   "selected_format": summ["selected_format"], "exhaustive_best": summ["exhaustive_best"],
                   "selector": w.selector["kind"], "selected_params": summ["selected_params"], "tuning": w.tuning,
                   "step": "selector kernel + SpMV in the selected format, matrix and x resident in HBM",
                   "launch": ("the step's two kernels captured once as a CUDA graph, replayed every step"
                              if w.graph is not None else "the step's two kernels launched directly"),
                   "direct_launch_step_ms": eager_step_ms,
                   "step_ms_after_write_only_flush": dirty_ms,
                   "l2": flush.describe(),
                   "parallelism": ("one GPU" if world == 1 else
                                   f"row blocks x{world}: nnz-balanced rows per rank, x broadcast from rank 0, each "
                                   f"rank's y slice on its own GPU (rank 0 rows {w.rows[0]}..{w.rows[1]})")},
        "roofline": summ["roofline"],
        "e2e": {"value": e2e_value, "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * a.n * world,
                "d2h_bytes_per_step": 8 * w.total_rows, "ms_per_step": e2e_ms, "steps": n_e2e,
                "windows_ms_per_step": e2e_windows, "of": "the median of three windows of `steps` steps",
                "copies": "spmv_run_host: pinned host x in and y out every step, through two device staging "
                          "pairs and two copy streams of the library (overlapping the neighbouring steps' "
                          "compute)", "y_matches_device_run": e2e_same},
        "gpu_launches": world * args.steps * (SELECT_LAUNCHES + launches_per_run(w.chosen, w.info_c)),
        "clocks": clocks,
        "formats": w.per_fmt,
        "selector": dict(w.selector, per_step_agrees=agree),
        "conversion_ms": w.conv_ms, "conversion_first_ms": w.conv_first_ms,
        "wall_s_timed_region": t_wall,
        "check": check,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(a, xh, args.cpu_seconds)
    del w
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and extras:
        line["extra_workloads"] = {e: measure_extra(e, args, sp, torch, stream, flush, model) for e in extras}
    if rank == 0 and world == 1 and args.batch_extra > 0:
        bw = BatchWorkload(args.batch_extra, args, 0, tune=False)
        cmp = bw.compare(max(10, min(args.steps, 100)), 3)
        cmp.pop("t_fam")
        cmp.pop("t_one")
        cmp["check_first_8_within_bound"] = bw.check()
        cmp["what"] = (f"the first {args.batch_extra} matrices of the batched configuration, formats from the batch "
                       f"selector with default parameters: the family kernels, the one-launch kernel and "
                       f"{args.batch_extra} separate launches, each replayed from a CUDA graph, L2 flushed")
        line.setdefault("extra_workloads", {})[f"batch{args.batch_extra}"] = cmp
        del bw
        bw = BatchWorkload(args.batch_extra, args, 0, tune=False, mixed=True)
        cmp = bw.compare(max(10, min(args.steps, 100)), 3)
        cmp.pop("t_fam")
        cmp.pop("t_one")
        cmp["check_first_8_within_bound"] = bw.check()
        cmp["what"] = (f"the same {args.batch_extra} matrices, matrix j in format j mod 5 (CSR, CSR5, ELL, SELL, HYB) "
                       f"with default parameters: family kernels against the one-launch kernel on a mixed batch")
        line["extra_workloads"][f"batch{args.batch_extra}_mixed"] = cmp
        del bw
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
