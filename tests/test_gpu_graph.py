"""The product and the selector under CUDA-graph capture: a step (selection
into a device buffer, then y = A x) captured once and replayed gives, every
replay, the y of a direct launch bit for bit and the same format id, in every
format, including the CSR and CSR5 row joins whose counters must be reset
by each run."""
import numpy as np
import pytest

import synth
from gpu_util import bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


def _mats():
    lens = np.array([0, 352, 352, 351, 1, 353, 704, 1, 0, 351, 353, 351, 354, 0, 5000, 3, 0], dtype=np.int32)
    return [
        synth.powerlaw(20_000, 301, xmax=3000, lmax=3000),
        synth.from_lengths_random_cols(lens, 7000, 302, "tile_edges_long"),
        synth.stencil(synth.STENCIL_27PT_3D, 13, 11, 7, 303),
    ]


@pytest.mark.parametrize("fmt", range(5))
def test_graph_replay_matches_direct_launch(sp, fmt):
    model = sp.Model.load(sp.MODEL_PATH)
    for a in _mats():
        d = sp.DeviceCSR.from_host(a)
        h = sp.spmv_convert(fmt, d)
        x = torch.as_tensor(synth.vector(a.n, 77)).cuda()
        fmt_direct = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        sp.spmv_select_async(d, model, fmt_direct)
        y_direct = sp.spmv_run(h, x)
        torch.cuda.synchronize()
        y = torch.empty(a.m, dtype=torch.float64, device="cuda")
        fmt_g = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # one run off the capture, as graph capture wants
            sp.spmv_select_async(d, model, fmt_g)
            sp.spmv_run(h, x, y)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sp.spmv_select_async(d, model, fmt_g)
            sp.spmv_run(h, x, y)
        for _ in range(3):
            y.fill_(float("nan"))
            fmt_g.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(bits(y.cpu().numpy()), bits(y_direct.cpu().numpy())), (a.name, sp.FORMATS[fmt])
            assert int(fmt_g.item()) == int(fmt_direct.item()), a.name
