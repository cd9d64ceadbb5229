"""Products with x and y in host memory through spmv_run_host (include/spmv.h):
every call's y against the oracle and bit for bit against spmv_run on device
buffers, with a different x on every call so that a copy overtaken by its
product, or a staging pair reused too early, would show."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
INVALID_ARG = -1  # spmv_status (include/spmv.h)


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


MATS = {
    "powerlaw": lambda: synth.powerlaw(30_000, 5),
    "stencil": lambda: synth.stencil(synth.STENCIL_27PT_3D, 24, 24, 24, seed=3),
    "wide": lambda: synth.from_lengths_random_cols(np.full(500, 9, np.int32), 40_000, 7, "wide"),
}


@pytest.mark.parametrize("fmt,params", [(0, None), (1, None), (2, None), (3, None), (3, {"sell_sigma": 1}),
                                        (3, {"sell_panel_cols": 7000}), (4, None)])
@pytest.mark.parametrize("name", sorted(MATS))
def test_run_host_every_call(sp, name, fmt, params):
    a = MATS[name]()
    d = sp.DeviceCSR.from_host(a)
    h = sp.spmv_convert(fmt, d, params)
    io = sp.HostIO(h)
    n_calls = 7
    xs = [torch.as_tensor(synth.vector(a.n, 100 + i)).pin_memory() for i in range(n_calls)]
    ys = [torch.empty(a.m, dtype=torch.float64).pin_memory() for _ in range(n_calls)]
    for i in range(n_calls):
        io.run(xs[i], ys[i])
    io.sync()
    for i in range(n_calls):
        x = xs[i].numpy()
        y = ys[i].numpy()
        y_dev = sp.spmv_run(h, xs[i].cuda()).cpu().numpy()
        assert np.array_equal(bits(y), bits(y_dev)), i
        assert np.all(np.abs(y - oracle.csr_spmv(a, x)) <= oracle.fp_bound(a, x)), i


def test_run_host_integer_exact_and_done_event(sp):
    """Integer values: y equals the oracle's bit for bit; `done` marks y ready."""
    a = synth.with_integer_values(synth.powerlaw(20_000, 9), 4)
    h = sp.spmv_convert(3, sp.DeviceCSR.from_host(a))
    io = sp.HostIO(h)
    x = torch.as_tensor(synth.integers(a.n, 5, -6, 6).astype(np.float64)).pin_memory()
    y = torch.empty(a.m, dtype=torch.float64).pin_memory()
    done = torch.cuda.Event()
    io.run(x, y, done=done)
    done.synchronize()
    assert np.array_equal(bits(y.numpy()), bits(oracle.csr_spmv(a, x.numpy())))


def test_run_host_reused_buffers_and_pageable_memory(sp):
    """One pair of host buffers rewritten between calls (waiting on `done`
    first), and pageable (unpinned) host memory."""
    a = synth.powerlaw(10_000, 13)
    h = sp.spmv_convert(0, sp.DeviceCSR.from_host(a))
    io = sp.HostIO(h)
    x = torch.empty(a.n, dtype=torch.float64)
    y = torch.empty(a.m, dtype=torch.float64)
    done = torch.cuda.Event()
    for i in range(4):
        x.copy_(torch.as_tensor(synth.vector(a.n, 50 + i)))
        io.run(x, y, done=done)
        done.synchronize()
        xn = x.numpy()
        assert np.all(np.abs(y.numpy() - oracle.csr_spmv(a, xn)) <= oracle.fp_bound(a, xn)), i


def test_run_host_refuses_bad_arguments(sp):
    a = synth.powerlaw(1000, 2)
    h = sp.spmv_convert(0, sp.DeviceCSR.from_host(a))
    io = sp.HostIO(h)
    with pytest.raises(ValueError):
        io.run(torch.empty(a.n + 1, dtype=torch.float64), torch.empty(a.m, dtype=torch.float64))
    with pytest.raises(ValueError):
        io.run(torch.empty(a.n, dtype=torch.float64).cuda(), torch.empty(a.m, dtype=torch.float64))
    lib = sp.lib()
    y = torch.empty(a.m, dtype=torch.float64)
    import ctypes

    assert lib.spmv_run_host(io._io, None, ctypes.c_void_p(y.data_ptr()), None, None) == INVALID_ARG
    assert lib.spmv_run_host(None, None, None, None, None) == INVALID_ARG
    out = ctypes.c_void_p()
    assert lib.spmv_host_io_create(None, ctypes.byref(out)) == INVALID_ARG
