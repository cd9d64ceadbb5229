"""GPU parity of the batched persistent launch (and its per-matrix comparison graph)."""
import numpy as np
import pytest

import synth
from gpu_util import bits, within_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


def _mats(n):
    out = []
    for j in range(n):
        out.append(synth.batch_matrix(j, r_lo=200, r_hi=20_000))
    lens = np.array([0, 0, 9000, 0, 3, 0, 0, 70, 1, 0] * 30, np.int32)
    out.append(synth.from_lengths_random_cols(lens, 10_000, 99, "empty_long"))
    return out


@pytest.mark.parametrize("params", [None, {"csr5_sigma": 4, "sell_C": 128, "sell_sigma": 256, "hyb_k": 2},
                                    {"csr_block_nnz": -8}, {"csr_block_nnz": 352}])
def test_batch_matches_single_runs(sp, params):
    mats = _mats(23)
    handles, xs, ys, ys2, singles = [], [], [], [], []
    for j, a in enumerate(mats):
        fmt = j % 5
        h = sp.spmv_convert(fmt, sp.DeviceCSR.from_host(a), params)
        x = torch.as_tensor(synth.vector(a.n, 500 + j)).cuda()
        handles.append(h)
        xs.append(x)
        ys.append(torch.full((a.m,), np.nan, dtype=torch.float64, device="cuda"))
        ys2.append(torch.full((a.m,), np.nan, dtype=torch.float64, device="cuda"))
        singles.append(sp.spmv_run(h, x).cpu().numpy())
    b = sp.Batch(handles)
    for rep in range(3):  # replays reuse counters and scratch
        b.run(xs, ys)
        b.run_separate(xs, ys2)
        torch.cuda.synchronize()
        for j, a in enumerate(mats):
            y = ys[j].cpu().numpy()
            assert np.array_equal(bits(y), bits(singles[j])), (j, rep)
            assert np.array_equal(bits(ys2[j].cpu().numpy()), bits(singles[j])), (j, rep)
            ok, msg = within_bound(a, xs[j].cpu().numpy(), y)
            assert ok, (j, msg)


def test_batch_new_vectors(sp):
    mats = _mats(6)
    handles = [sp.spmv_convert(j % 5, sp.DeviceCSR.from_host(a)) for j, a in enumerate(mats)]
    b = sp.Batch(handles)
    for seed in (1, 2):
        xs = [torch.as_tensor(synth.vector(a.n, seed * 100 + j)).cuda() for j, a in enumerate(mats)]
        ys = [torch.empty(a.m, dtype=torch.float64, device="cuda") for a in mats]
        b.run(xs, ys)
        torch.cuda.synchronize()
        for j, a in enumerate(mats):
            ok, msg = within_bound(a, xs[j].cpu().numpy(), ys[j].cpu().numpy())
            assert ok, (seed, j, msg)


def test_batch_refuses_sell_in_column_panels(sp):
    a = _mats(1)[0]
    h = sp.spmv_convert(3, sp.DeviceCSR.from_host(a), {"sell_panel_cols": 50})
    assert h.info()["aux"][3] > 1
    with pytest.raises(sp.SpmvError) as ei:
        sp.Batch([h])
    assert ei.value.name == "INVALID_ARG"
