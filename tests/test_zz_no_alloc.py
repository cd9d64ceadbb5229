"""The allocation-free entry point against the ordinary one and the oracle.

spmv_csr_run_noalloc serves callers that cannot call cudaMalloc when they need
a product: code under a memory manager that has already reserved every device
byte, or latency-critical paths that must not enter the CUDA allocator (its
calls can synchronise the device).  It keeps its scratch in a static device
array of the library.  Two calls in a row (the second reusing the array the
first left behind) must each match spmv_run on a converted handle and the CPU
oracle within the FP64 tolerance used throughout the tests, and, on
integer-valued inputs, both bit for bit.  The file name sorts last so a run
that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


def _cases():
    lens = np.array([0, 0, 9000, 0, 3, 0, 0, 70, 1, 0] * 30, np.int32)
    return [synth.config1(), synth.powerlaw(30_000, 11, xmax=3000, lmax=3000),
            synth.from_lengths_random_cols(lens, 10_000, 12, "empty_long"), synth.tiny_random(5, 4, 0.5, 13),
            synth.CSR(100, 7, np.zeros(101, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty")]


@pytest.mark.parametrize("ci", range(5))
def test_noalloc_matches_spmv_run_twice(sp, ci):
    a = _cases()[ci]
    d = sp.DeviceCSR.from_host(a)
    h = sp.spmv_convert(sp.SPMV_CSR, d)
    bound = None
    for call in range(2):
        xh = synth.vector(a.n, 40 + call)
        x = torch.as_tensor(xh).cuda()
        y_ref = sp.spmv_run(h, x).cpu().numpy()
        y = torch.full((a.m,), np.nan, dtype=torch.float64, device="cuda")
        sp.spmv_csr_run_noalloc(d, x, y)
        y = y.cpu().numpy()
        bound = oracle.fp_bound(a, xh)
        assert np.all(np.abs(y - y_ref) <= bound), (a.name, call, float(np.max(np.abs(y - y_ref) - bound)))
        y_or = oracle.csr_spmv(a, xh)
        assert np.all(np.abs(y - y_or) <= bound), (a.name, call, float(np.max(np.abs(y - y_or) - bound)))


@pytest.mark.parametrize("ci", range(5))
def test_noalloc_integer_values_bit_exact_twice(sp, ci):
    """Small integer values and x: every summation order gives the exact row
    sums, so y equals the oracle's and spmv_run's bit for bit."""
    a = synth.with_integer_values(_cases()[ci], 60 + ci)
    d = sp.DeviceCSR.from_host(a)
    h = sp.spmv_convert(sp.SPMV_CSR, d)
    for call in range(2):
        xh = synth.integers(a.n, 70 + ci + 10 * call, -16, 16)
        x = torch.as_tensor(xh).cuda()
        y = torch.full((a.m,), np.nan, dtype=torch.float64, device="cuda")
        sp.spmv_csr_run_noalloc(d, x, y)
        y = y.cpu().numpy()
        assert np.array_equal(y.view(np.int64), oracle.csr_spmv(a, xh).view(np.int64)), (a.name, call)
        assert np.array_equal(y.view(np.int64), sp.spmv_run(h, x).cpu().numpy().view(np.int64)), (a.name, call)


def test_noalloc_rejects_oversize(sp):
    a = synth.config1()
    d = sp.DeviceCSR.from_host(a)
    big = sp._abi.spmv_csr(a.m, a.n, (1 << 29) + 1, d.ptr.data_ptr(), d.idx.data_ptr(), d.val.data_ptr())
    x = torch.zeros(a.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(a.m, dtype=torch.float64, device="cuda")
    import ctypes

    rc = sp.lib().spmv_csr_run_noalloc(ctypes.byref(big), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), None)
    assert rc == -3 and b"at most" in sp.lib().spmv_last_error()
