"""Parity at the workloads' full sizes, in the configurations bench.py times,
on sampled rows the oracle computes one by one.

  * 27-point stencil on 224^3 (300.8 M nonzeros): HYB, ELL and SELL (the
    selector's pick).
  * 2e7-row power-law graph (239 M nonzeros): SELL in its automatic column
    panels (x is 160 MB) and CSR5.
  * the 512-matrix batch with the formats the batch model picks: every
    matrix's y from the persistent launches equals its own product bit for
    bit, and sampled rows of every matrix are within the FP64 bound.
"""
import numpy as np
import pytest

import synth
from gpu_util import bits, row_subset, within_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


def _sample_rows(a, k=4096, extra=64):
    lens = np.diff(a.ptr)
    picks = [np.linspace(0, a.m - 1, k).astype(np.int64), np.argsort(lens, kind="stable")[-extra:],
             np.argsort(lens, kind="stable")[:extra]]
    return np.unique(np.concatenate(picks))


def _check(sp, a, x, fmt, params=None):
    d = sp.DeviceCSR.from_host(a)
    h = sp.spmv_convert(fmt, d, params)
    y = sp.spmv_run(h, torch.as_tensor(x).cuda()).cpu().numpy()
    rows = _sample_rows(a)
    ok, msg = within_bound(row_subset(a, rows), x, y[rows])
    info = h.info()
    del h, d
    torch.cuda.empty_cache()
    return ok, msg, info


def test_stencil_224_sampled_rows(sp):
    a = synth.config5_stencil()
    x = synth.vector(a.n, 1)
    for fmt in (sp.SPMV_HYB, sp.SPMV_ELL, sp.SPMV_SELL):
        ok, msg, _ = _check(sp, a, x, fmt)
        assert ok, f"{sp.FORMATS[fmt]}: {msg}"


def test_graph_2e7_sampled_rows(sp):
    a = synth.config5_graph()
    x = synth.vector(a.n, 1)
    ok, msg, info = _check(sp, a, x, sp.SPMV_SELL)
    assert info["aux"][3] == 3, info  # x of 160 MB: three column panels
    assert ok, f"SELL in panels: {msg}"
    ok, msg, _ = _check(sp, a, x, sp.SPMV_CSR5)
    assert ok, f"CSR5: {msg}"


def test_batch512_sampled_rows(sp):
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
    b = sp.Batch(handles)
    b.run(xs, ys)
    torch.cuda.synchronize()
    for j, (a, h) in enumerate(zip(mats, handles)):
        y = ys[j].cpu().numpy()
        single = sp.spmv_run(h, xs[j]).cpu().numpy()
        assert np.array_equal(bits(y), bits(single)), j
        rows = _sample_rows(a, k=64, extra=8)
        ok, msg = within_bound(row_subset(a, rows), xs[j].cpu().numpy(), y[rows])
        assert ok, (j, msg)
