"""Randomised parity sweep: seeded random matrices whose row lengths mix the
cases the kernels split on (empty rows, single entries, rows just below and
above the CSR tile width of 352 and the CSR5 tile of 1024, long rows spanning
many tiles), in every format under several parameter sets.  Integer values
make every format's y bit-identical to the oracle's; every handle's way back
to CSR is exact."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PARAMS = {
    0: [None, {"csr_block_nnz": 352}, {"csr_block_nnz": -4}, {"csr_block_nnz": -16}],
    1: [None, {"csr5_sigma": 3}, {"csr5_sigma": 17}],
    2: [None],
    3: [None, {"sell_C": 64, "sell_sigma": 128}, {"sell_C": 128, "sell_sigma": 1}, {"sell_panel_cols": 97},
        {"sell_C": 64, "sell_panel_cols": 1000}],
    4: [None, {"hyb_k": 2}, {"hyb_k": -1}],
}
SPECIAL = np.array([0, 1, 2, 31, 32, 33, 351, 352, 353, 703, 704, 705, 1023, 1024, 1025, 3000], np.int64)


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


def _matrix(seed):
    rng = np.random.default_rng(1000 + seed)
    m = int(rng.integers(1, 3000))
    n = int(rng.integers(1, 4000))
    law = seed % 3
    if law == 0:  # mostly empty rows with a few special lengths
        lens = np.where(rng.random(m) < 0.7, 0, rng.choice(SPECIAL, size=m))
    elif law == 1:  # short rows with special lengths sprinkled in
        lens = rng.integers(0, 5, size=m)
        pick = rng.random(m) < 0.05
        lens[pick] = rng.choice(SPECIAL, size=int(pick.sum()))
    else:  # heavy-tailed
        lens = np.minimum(np.floor(rng.pareto(1.2, size=m) * 3).astype(np.int64), 5000)
    lens = np.minimum(lens, 8 * n)  # duplicates allowed, but keep rows finite
    lens = np.minimum(lens, 200_000 // max(m, 1) + SPECIAL.max()).astype(np.int64)
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    nnz = int(ptr[-1])
    idx = rng.integers(0, n, size=nnz).astype(np.int32)  # unsorted, duplicates possible
    val = rng.integers(-8, 9, size=nnz).astype(np.float64)
    return synth.CSR(m, n, ptr, idx, val, f"random{seed}")


@pytest.mark.parametrize("seed", range(120))
def test_random_matrices_every_format(sp, seed):
    a = _matrix(seed)
    x = np.random.default_rng(seed).integers(-16, 17, size=a.n).astype(np.float64)
    ref = oracle.csr_spmv(a, x)
    d = sp.DeviceCSR.from_host(a)
    xd = torch.as_tensor(x).cuda()
    for fmt, plist in PARAMS.items():
        for p in plist:
            try:
                h = sp.spmv_convert(fmt, d, p)
            except sp.SpmvError as e:  # ELL of a matrix with one very long row may exceed the cap
                assert fmt == 2 and e.name == "TOO_LARGE", (fmt, p, e.name)
                continue
            y = sp.spmv_run(h, xd).cpu().numpy()
            assert np.array_equal(bits(y), bits(ref)), (a.name, sp.FORMATS[fmt], p)
            pt, it, vt = (t.cpu().numpy() for t in sp.spmv_to_csr(h))
            assert np.array_equal(pt, a.ptr) and np.array_equal(it, a.idx) and np.array_equal(bits(vt), bits(a.val)), \
                (a.name, sp.FORMATS[fmt], p)


@pytest.mark.parametrize("seed", range(24))
def test_random_matrices_features(sp, seed):
    """The 16 features of random matrices around the sampling boundary (8192
    rows), with empty rows and rows past the 512 length cap, against the oracle."""
    rng = np.random.default_rng(5000 + seed)
    m = int(rng.choice([1, 7, 8191, 8192, 8193, 20_000, int(rng.integers(2, 60_000))]))
    n = int(rng.integers(1, 100_000))
    lens = np.where(rng.random(m) < 0.2, 0, rng.integers(1, 40, size=m))
    lens[rng.random(m) < 0.01] = 700
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    a = synth.CSR(m, n, ptr, rng.integers(0, n, size=int(ptr[-1])).astype(np.int32), np.ones(int(ptr[-1])),
                  f"feat{seed}")
    f = sp.spmv_features(sp.DeviceCSR.from_host(a)).cpu().numpy()
    ref = oracle.features(a).astype(np.float32)
    assert np.allclose(f, ref, rtol=2e-6, atol=0), (a.name, np.stack([f, ref]))


@pytest.mark.parametrize("seed", range(8))
def test_features_cluster_sizes_and_unaligned_idx(sp, seed):
    """The features kernel's two cluster sizes (8 and 16 CTAs), and its scalar
    index loads (idx not 16-byte aligned) beside the 16-byte ones, give the
    same features bit for bit and the same selection, within the oracle's
    tolerance."""
    rng = np.random.default_rng(7000 + seed)
    m = int(rng.choice([5, 8191, 8192, 8193, int(rng.integers(9000, 80_000))]))
    n = int(rng.integers(1, 100_000))
    lens = np.where(rng.random(m) < 0.2, 0, rng.integers(1, 40, size=m))
    lens[rng.random(m) < 0.01] = 700
    lens[-1] = 3  # the last row ends at the end of idx: its 16-byte words run past it
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    a = synth.CSR(m, n, ptr, rng.integers(0, n, size=int(ptr[-1])).astype(np.int32), np.ones(int(ptr[-1])),
                  f"cluster{seed}")
    d = sp.DeviceCSR.from_host(a)
    idx_pad = torch.zeros(a.nnz + 1, dtype=torch.int32, device="cuda")
    idx_pad[1:] = d.idx
    du = sp.DeviceCSR(a.m, a.n, d.ptr, idx_pad[1:], d.val)
    assert du.idx.data_ptr() % 16 != 0
    model = sp.Model.load(sp.MODEL_PATH)
    outs, sels = [], []
    try:
        for ctas in (0, 8, 16):
            sp.spmv_debug_features_cluster(ctas)
            for dd in (d, du):
                outs.append(sp.spmv_features(dd).cpu().numpy())
                sels.append(sp.spmv_select(dd, model))
    finally:
        sp.spmv_debug_features_cluster(0)
    for f in outs[1:]:
        assert np.array_equal(f.view(np.uint32), outs[0].view(np.uint32)), (a.name, np.stack([f, outs[0]]))
    assert len(set(sels)) == 1, sels
    ref = oracle.features(a).astype(np.float32)
    assert np.allclose(outs[0], ref, rtol=2e-6, atol=0), (a.name, np.stack([outs[0], ref]))
