"""The row-partitioned product (one product split over ranks by nnz-balanced
row blocks, x replicated, y gathered), on CPU with gloo.

Each rank runs its block through the same per-rank code as on the GPU, with
the oracle as the per-rank computer; the gathered y must equal the oracle's
product of the whole matrix bit for bit on integer-valued inputs (every
summation order is exact there, and each row is summed by one rank).
"""
import json
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import synth
from paper_1805_11938_gb300.distributed import local_csr, row_partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle, synth
    from paper_1805_11938_gb300.distributed import RowPartitioned
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    out = []
    for case in {cases!r}:
        if case == "powerlaw":
            a = synth.with_integer_values(synth.powerlaw(3001, 5, xmax=400, lmax=400), 6)
        elif case == "empty_rows":
            lens = np.array([0, 0, 90, 0, 3, 0, 0, 7, 1, 0] * 40, np.int32)
            a = synth.with_integer_values(synth.from_lengths_random_cols(lens, 500, 7, "e"), 8)
        else:  # fewer rows than ranks
            a = synth.with_integer_values(synth.from_lengths_random_cols(np.array([5, 0], np.int32), 9, 9, "t"), 10)
        x = torch.from_numpy(synth.integers(a.n, 11, -9, 9)) if rank == 0 else torch.zeros(a.n, dtype=torch.float64)
        rp = RowPartitioned(a, rank, world, dist,
                            multiply=lambda blk, xv: torch.from_numpy(oracle.csr_spmv(blk, xv.numpy())))
        rp.broadcast_x(x)  # x replicated from rank 0
        y = rp.gather_y(rp.run(x))
        ref = oracle.csr_spmv(a, synth.integers(a.n, 11, -9, 9))
        out.append({{"case": case, "rows": rp.rows, "block_nnz": rp.block.nnz,
                     "same": bool(np.array_equal(y.numpy().view(np.int64), ref.view(np.int64)))}})
    dist.barrier()
    dist.destroy_process_group()
    print(json.dumps(out), flush=True)
""")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(tmp_path, world, cases):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT, cases=cases))
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    return outs


@pytest.mark.parametrize("world", [2, 3])
def test_row_partitioned_product_gloo(tmp_path, world):
    pytest.importorskip("torch.distributed")
    cases = ["powerlaw", "empty_rows", "fewer_rows_than_ranks"]
    outs = _run(tmp_path, world, cases)
    for r, o in enumerate(outs):
        for c in o:
            assert c["same"], (world, r, c)
    # two rows (5 nonzeros, then none) over 2 or 3 ranks: blocks as row_partition gives them
    rows = [o[2]["rows"] for o in outs]
    assert rows == np.diff(row_partition([0, 5, 5], world)).tolist() and sum(rows) == 2
    assert [o[2]["block_nnz"] for o in outs].count(5) == 1


def test_row_partition_balances_nonzeros():
    """Blocks cover the rows in order; each holds nnz / parts nonzeros up to one row."""
    a = synth.powerlaw(20_000, 3, xmax=3000, lmax=3000)
    lens = np.diff(a.ptr)
    for parts in (1, 2, 3, 8, 64):
        b = row_partition(a.ptr, parts)
        assert b[0] == 0 and b[-1] == a.m and np.all(np.diff(b) >= 0)
        block_nnz = np.diff(a.ptr[b].astype(np.int64))
        assert block_nnz.sum() == a.nnz
        assert np.all(np.abs(block_nnz - a.nnz / parts) <= lens.max()), (parts, block_nnz)
    # the paper's Table I matrix (ptr 0, 2, 5, 6, 8) in two blocks: rows 0-1 (5 nonzeros), rows 2-3 (3)
    assert row_partition([0, 2, 5, 6, 8], 2).tolist() == [0, 2, 4]
    assert row_partition([0, 0, 0, 0], 3).tolist() == [0, 1, 2, 3]  # no nonzeros: rows split evenly
    assert row_partition([0, 10], 3).tolist() == [0, 1, 1, 1]


def test_local_csr_is_the_row_block():
    a = synth.powerlaw(500, 4, xmax=50, lmax=50)
    blk = local_csr(a, 100, 230)
    assert blk.m == 130 and blk.n == a.n and blk.ptr[0] == 0
    for i in range(130):
        r = 100 + i
        assert np.array_equal(blk.idx[blk.ptr[i]:blk.ptr[i + 1]], a.idx[a.ptr[r]:a.ptr[r + 1]])
        assert np.array_equal(blk.val[blk.ptr[i]:blk.ptr[i + 1]], a.val[a.ptr[r]:a.ptr[r + 1]])
