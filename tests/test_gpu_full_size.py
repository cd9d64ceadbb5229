"""Parity at the workloads' full sizes, in the configurations bench.py times.

Every row of y is compared with the oracle (its rows split over the host
cores, bit-identical to its single-threaded loop) within the FP64 bound, and
every conversion's way back to CSR with the input, bit for bit (ptr, column
order, value bits).

  * power-law n = 2e6 (13.8 M nonzeros): all five formats, with the
    autotuner's grid (CSR tiles, CSR5 sigma 16/24/32, SELL C = 32/64/128),
    ELL at the benchmark's 160 GiB cap (its padded layout is about 119 GB).
  * 27-point stencil on 224^3 (300.8 M nonzeros): all five formats, SELL at
    C = 32/64/128 and at C = 64 with sigma = 1 (rows in place, no perm read).
  * power-law graph n = 2e7 (239 M nonzeros): CSR, CSR5, HYB, SELL in its
    automatic column panels (x is 160 MB) and in one panel; ELL refused.
  * the 512-matrix batch with the formats the batch model picks, in both
    persistent ways: every matrix's y equals its own product bit for bit,
    and every row of every matrix is within the FP64 bound.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ELL_CAP = 160 << 30  # bench.py's --ell-cap-gb default


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


def _cores():
    return max(1, len(os.sched_getaffinity(0)))


def _all_rows(sp, a, x, cases, seed_note):
    """Runs every (format, params) case on the full matrix; returns the list of
    failures (empty when every row is within the bound and every round trip
    is exact) and the handles' info."""
    y_ref = oracle.csr_spmv_threads(a, x, _cores())
    bound = oracle.fp_bound(a, x)
    d = sp.DeviceCSR.from_host(a)
    xd = torch.as_tensor(x).cuda()
    fails, infos = [], []
    for fmt, params in cases:
        tag = f"{sp.FORMATS[fmt]} {params or 'default'} ({seed_note})"
        h = sp.spmv_convert(fmt, d, params)
        infos.append((fmt, params, h.info()))
        y = sp.spmv_run(h, xd).cpu().numpy()
        err = np.abs(y - y_ref)
        bad = ~(err <= bound)
        if bad.any():
            i = int(np.argmax(bad))
            fails.append(f"{tag}: {int(bad.sum())} rows off, row {i}: y={y[i]!r} ref={y_ref[i]!r} bound={bound[i]:.3e}")
        p, ii, v = sp.spmv_to_csr(h)
        if not (torch.equal(p, d.ptr) and torch.equal(ii, d.idx) and torch.equal(v.view(torch.int64), d.val.view(torch.int64))):
            fails.append(f"{tag}: round trip differs")
        del h, p, ii, v
        torch.cuda.empty_cache()
    del d, xd
    torch.cuda.empty_cache()
    return fails, infos


def test_power_law_2e6_all_rows_every_format(sp):
    a = synth.config2()
    x = synth.vector(a.n, 1)
    cases = [(0, None), (0, {"csr_block_nnz": 352}), (1, None), (1, {"csr5_sigma": 16}), (1, {"csr5_sigma": 24}),
             (2, {"max_bytes": ELL_CAP}), (3, None), (3, {"sell_C": 32, "sell_sigma": 1024}), (3, {"sell_C": 64}),
             (3, {"sell_C": 128}), (4, None)]
    fails, infos = _all_rows(sp, a, x, cases, "power-law 2e6")
    assert not fails, fails
    ell = [i for f, _, i in infos if f == 2][0]
    assert ell["stored_slots"] == a.m * int(np.diff(a.ptr).max())  # the full padded layout was checked


def test_stencil_224_all_rows_every_format(sp):
    a = synth.config5_stencil()
    x = synth.vector(a.n, 1)
    cases = [(0, None), (1, None), (2, None), (3, None), (3, {"sell_C": 64}), (3, {"sell_C": 64, "sell_sigma": 1}),
             (3, {"sell_C": 128}), (4, None)]
    fails, _ = _all_rows(sp, a, x, cases, "stencil 224^3")
    assert not fails, fails


def test_graph_2e7_all_rows(sp):
    a = synth.config5_graph()
    x = synth.vector(a.n, 1)
    cases = [(3, None), (3, {"sell_panel_cols": -1}), (1, None), (0, None), (4, None)]
    fails, infos = _all_rows(sp, a, x, cases, "graph 2e7")
    assert not fails, fails
    assert infos[0][2]["aux"][3] == 3, infos[0][2]  # x of 160 MB: three column panels
    d = sp.DeviceCSR.from_host(a)
    with pytest.raises(sp.SpmvError) as ei:
        sp.spmv_convert(sp.SPMV_ELL, d)
    assert ei.value.name == "TOO_LARGE"


@pytest.mark.parametrize("one_launch", [False, True])
def test_batch512_all_rows(sp, one_launch):
    """The 512-matrix batch in the batch model's formats, both persistent ways:
    every matrix's y equals its own product bit for bit, and every row of every
    matrix is within the bound of the oracle's."""
    model = sp.Model.load(sp.MODEL_BATCH_PATH)
    handles, xs, ys, mats = [], [], [], []
    for j in range(512):
        a = synth.batch_matrix(j)
        d = sp.DeviceCSR.from_host(a)
        handles.append(sp.spmv_convert(sp.spmv_select(d, model), d))
        xs.append(torch.as_tensor(synth.vector(a.n, 900 + j)).cuda())
        ys.append(torch.empty(a.m, dtype=torch.float64, device="cuda"))
        mats.append(a)
        del d
    b = sp.Batch(handles, one_launch=one_launch)
    b.run(xs, ys)
    torch.cuda.synchronize()
    for j, (a, h) in enumerate(zip(mats, handles)):
        y = ys[j].cpu().numpy()
        single = sp.spmv_run(h, xs[j]).cpu().numpy()
        assert np.array_equal(bits(y), bits(single)), j
        x = xs[j].cpu().numpy()
        ref = oracle.csr_spmv_threads(a, x, _cores())
        bound = oracle.fp_bound(a, x)
        bad = ~(np.abs(y - ref) <= bound)
        assert not bad.any(), (j, int(np.argmax(bad)))
