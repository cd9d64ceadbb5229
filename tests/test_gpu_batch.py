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


@pytest.mark.parametrize("one_launch", [False, True])
@pytest.mark.parametrize("params", [None, {"csr5_sigma": 4, "sell_C": 128, "sell_sigma": 256, "hyb_k": 2},
                                    {"csr_block_nnz": -8}, {"csr_block_nnz": 352},
                                    {"sell_C": 64, "sell_sigma": 1}])  # SELL rows in place: run writes y without perm
def test_batch_matches_single_runs(sp, params, one_launch):
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
    b = sp.Batch(handles, one_launch=one_launch)
    if one_launch:  # one kernel, plus the HYB tails' own when there are any
        tails = any(h.info()["fmt"] == 4 and h.info()["aux"][1] > 0 for h in handles)
        assert b.launches() == 1 + tails
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


def test_batch_one_launch_mixed_sell_heights(sp):
    """SELL matrices of all three slice heights in one launch (the height picked
    per task at run time): bit for bit each matrix's own product."""
    mats = _mats(12)
    handles = [sp.spmv_convert(3, sp.DeviceCSR.from_host(a), {"sell_C": (32, 64, 128)[j % 3]})
               for j, a in enumerate(mats)]
    xs = [torch.as_tensor(synth.vector(a.n, 700 + j)).cuda() for j, a in enumerate(mats)]
    singles = [sp.spmv_run(h, x).cpu().numpy() for h, x in zip(handles, xs)]
    b = sp.Batch(handles, one_launch=True)
    assert b.launches() == 1
    assert sp.Batch(handles).launches() == 3  # the family kernels: one per slice height
    ys = [torch.full((a.m,), np.nan, dtype=torch.float64, device="cuda") for a in mats]
    for rep in range(2):
        b.run(xs, ys)
        torch.cuda.synchronize()
        for j in range(len(mats)):
            assert np.array_equal(bits(ys[j].cpu().numpy()), bits(singles[j])), (j, rep)
    import ctypes

    arr = (ctypes.c_void_p * 1)(handles[0].raw.value)
    out = ctypes.c_void_p()
    assert sp.lib().spmv_batch_build_ex(arr, 1, 2, None, ctypes.byref(out)) == -1  # unknown flag
    assert not out.value
