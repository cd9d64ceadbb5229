"""The multi-rank host path of bench.py, on CPU with gloo (world size 2).

Each rank multiplies its own row block of the one matrix (or its share of a
batch) and the ranks exchange only their timed totals: the slowest rank's
time (max) and the flops of all ranks (sum) give the whole-job rate.  The
reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    import bench
    rank = int(os.environ["RANK"])
    dist.init_process_group("gloo")
    # rank r: timed total 10 (r + 1) ms, flops 1e9 (r + 1) (ranks hold different shares)
    t, v = bench.reduce_over_ranks(10.0 * (rank + 1), 1e9 * (rank + 1), dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    print(json.dumps({{"rank": rank, "t": t, "v": v}}), flush=True)
""")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reduce_over_ranks_gloo_world2(tmp_path):
    pytest.importorskip("torch.distributed")
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["t"] == 20.0                      # the slowest rank's total
        assert o["v"] == pytest.approx(3e9 / 20e6)  # all ranks' flops over that time, GFLOP/s


def test_reduce_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench

    t, v = bench.reduce_over_ranks(4.0, 8e9)
    assert t == 4.0 and v == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    args = argparse.Namespace(workload="laplacian_64", steps=2, warmup=1)
    bench.run_reference(args, rank=1, world=2)  # a non-zero rank returns without work or output
    assert capsys.readouterr().out == ""
