"""GPU parity of the five formats against the CPU oracle, through the C ABI.

y: within |y_i - y_ref,i| <= 4 nnz_i 2^-53 sum_j |a_ij x_j| (integer-valued
inputs: bit-identical).  Conversions: byte-identical to the oracle's layouts
and an exact round trip back to CSR.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import bits, matrices_small, row_subset, within_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sp = None
probe = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global sp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m
    from paper_1805_11938_gb300 import probe as pr

    m.lib()
    sp = m
    globals()["probe"] = pr
    yield


MATS = matrices_small()
PARAMS = {
    0: [None, {"csr_block_nnz": 352}, {"csr_block_nnz": -2}, {"csr_block_nnz": -32}],
    1: [None, {"csr5_sigma": 1}, {"csr5_sigma": 4}, {"csr5_sigma": 32}],
    2: [None],
    3: [None, {"sell_C": 64, "sell_sigma": 1}, {"sell_C": 128, "sell_sigma": -1}, {"sell_C": 32, "sell_sigma": 256},
        {"sell_panel_cols": 700}, {"sell_C": 64, "sell_panel_cols": 1023}],
    4: [None, {"hyb_k": 1}, {"hyb_k": -1}],
}


def _run(a, fmt, params, x):
    d = sp.DeviceCSR.from_host(a)
    h = sp.spmv_convert(fmt, d, params)
    y = sp.spmv_run(h, torch.as_tensor(x).cuda()).cpu().numpy()
    return h, y


@pytest.mark.parametrize("fmt", range(5))
@pytest.mark.parametrize("mi", range(len(MATS)))
def test_product_within_bound(fmt, mi):
    a = MATS[mi]
    x = synth.vector(a.n, 1000 + mi)
    for p in PARAMS[fmt]:
        h, y = _run(a, fmt, p, x)
        ok, msg = within_bound(a, x, y)
        assert ok, f"{sp.FORMATS[fmt]} {p} on {a.name}: {msg}"
        y2 = sp.spmv_run(h, torch.as_tensor(x).cuda()).cpu().numpy()
        assert np.array_equal(bits(y), bits(y2)), "run is not deterministic"


@pytest.mark.parametrize("fmt", range(5))
def test_integer_inputs_bit_identical(fmt):
    for mi, a0 in enumerate(MATS):
        a = synth.with_integer_values(a0, 7 + mi)
        x = synth.integers(a.n, 8 + mi, -16, 16)
        ref = oracle.csr_spmv(a, x)
        for p in PARAMS[fmt]:
            _, y = _run(a, fmt, p, x)
            assert np.array_equal(bits(y), bits(ref)), f"{sp.FORMATS[fmt]} {p} on {a.name}"


@pytest.mark.parametrize("fmt", range(5))
@pytest.mark.parametrize("mi", range(len(MATS)))
def test_round_trip_exact(fmt, mi):
    a = MATS[mi]
    a = synth.CSR(a.m, a.n, a.ptr, a.idx, a.val.copy(), a.name)
    if a.nnz > 2:
        a.val[0] = -0.0
        a.val[-1] = 0.0  # explicit zero survives
    d = sp.DeviceCSR.from_host(a)
    for p in PARAMS[fmt]:
        h = sp.spmv_convert(fmt, d, p)
        ptr, idx, val = (t.cpu().numpy() for t in sp.spmv_to_csr(h))
        assert np.array_equal(ptr, a.ptr) and np.array_equal(idx, a.idx) and np.array_equal(bits(val), bits(a.val)), \
            f"{sp.FORMATS[fmt]} {p} on {a.name}"


def test_unsorted_columns_and_duplicates():
    ptr = np.array([0, 4, 4, 7], np.int32)
    idx = np.array([3, 1, 3, 0, 2, 2, 1], np.int32)
    val = np.array([1.5, -2.0, 4.0, 8.0, 1.0, 3.0, -1.0])
    a = synth.CSR(3, 4, ptr, idx, val, "dups")
    x = np.array([1.0, 2.0, 3.0, 4.0])
    ref = oracle.csr_spmv(a, x)
    for fmt in range(5):
        for p in PARAMS[fmt]:
            h, y = _run(a, fmt, p, x)
            assert np.array_equal(bits(y), bits(ref)), (fmt, p)
            pt, it, vt = (t.cpu().numpy() for t in sp.spmv_to_csr(h))
            assert np.array_equal(it, idx) and np.array_equal(vt, val)


def test_sell_panels_unsorted_columns_and_duplicates():
    """Column panels of one or a few columns: the product adds the panels in
    order and the way back restores every entry to its CSR position."""
    ptr = np.array([0, 4, 4, 7, 9], np.int32)
    idx = np.array([3, 1, 3, 0, 2, 2, 1, 0, 3], np.int32)
    val = np.array([1.5, -2.0, 4.0, 8.0, 1.0, 3.0, -1.0, -0.0, 0.0])
    a = synth.CSR(4, 4, ptr, idx, val, "dups")
    x = np.array([1.0, 2.0, 3.0, 4.0])
    ref = oracle.csr_spmv(a, x)
    for pc in (1, 2, 3):
        h, y = _run(a, 3, {"sell_panel_cols": pc}, x)
        info = h.info()
        assert info["aux"][3] == -(-4 // pc) and info["params"]["sell_panel_cols"] == pc
        assert np.array_equal(bits(y), bits(ref)), pc
        pt, it, vt = (t.cpu().numpy() for t in sp.spmv_to_csr(h))
        assert np.array_equal(pt, ptr) and np.array_equal(it, idx) and np.array_equal(bits(vt), bits(val)), pc


@pytest.mark.parametrize("pc,C,sigma", [(5000, 32, 0), (7001, 64, 1024), (2500, 128, 128), (5000, 32, 1)])
def test_sell_panels_share_one_row_order(pc, C, sigma):
    """Column panels keep one row order, so that partial sums stay in that
    order between panels: rows longer than 32 entries first, then the others
    in windows of min(sigma, 2^16) consecutive rows; inside each group, rows
    sorted, stably and descending, by their per-panel lengths taken
    lexicographically (panel 0 first).  The handle's perm is compared with
    numpy's stable lexsort of the keys counted on the host; y and the way back
    are exact on integer-valued inputs."""
    a = synth.with_integer_values(MATS[1], 55)  # power-law rows, 20000 x 20000
    x = synth.integers(a.n, 56, -7, 7)
    h, y = _run(a, 3, {"sell_panel_cols": pc, "sell_C": C, "sell_sigma": sigma}, x)
    P = -(-a.n // pc)
    assert h.info()["aux"][3] == P
    rows = np.repeat(np.arange(a.m), np.diff(a.ptr))
    lens = [np.bincount(rows[(a.idx // pc) == p], minlength=a.m) for p in range(P)]
    window = min(a.m if sigma == 0 else sigma, 1 << 16)
    group = np.where(np.diff(a.ptr) > 32, 0, 1 + np.arange(a.m) // window)
    order = np.lexsort(tuple(-l for l in reversed(lens)) + (group,))
    if sigma == 1:  # plain SELL: no sorting at all
        order = np.arange(a.m)
    assert np.array_equal(h.array("perm").cpu().numpy(), order)
    assert np.array_equal(bits(y), bits(oracle.csr_spmv(a, x)))
    pt, it, vt = (t.cpu().numpy() for t in sp.spmv_to_csr(h))
    assert np.array_equal(pt, a.ptr) and np.array_equal(it, a.idx) and np.array_equal(bits(vt), bits(a.val))


def test_sell_panel_count_is_bounded():
    """Panels are keys of the shared row order's sort, so their number is
    bounded: 300 panels are refused (INVALID_ARG), 200 convert and multiply."""
    lens = np.full(500, 4, np.int32)
    a = synth.with_integer_values(synth.from_lengths_random_cols(lens, 600, 19, "narrow"), 20)
    d = sp.DeviceCSR.from_host(a)
    with pytest.raises(sp.SpmvError) as ei:
        sp.spmv_convert(sp.SPMV_SELL, d, {"sell_panel_cols": 2})
    assert ei.value.name == "INVALID_ARG"
    x = synth.integers(a.n, 21, -5, 5)
    h, y = _run(a, 3, {"sell_panel_cols": 3}, x)
    assert h.info()["aux"][3] == 200
    assert np.array_equal(bits(y), bits(oracle.csr_spmv(a, x)))


def test_sell_panel_rule_splits_large_x():
    """x of 13e6 doubles (99 MiB, above 96 MiB) is split into panels of at most
    64 MiB of x; a smaller x stays in one panel."""
    lens = np.full(3000, 5, np.int32)
    a = synth.from_lengths_random_cols(lens, 13_000_000, 17, "wide")
    x = synth.vector(a.n, 18)
    h, y = _run(a, 3, None, x)
    info = h.info()
    assert info["aux"][3] == 2 and info["params"]["sell_panel_cols"] == 6_500_000
    ok, msg = within_bound(a, x, y)
    assert ok, msg
    h1, y1 = _run(a, 3, {"sell_panel_cols": -1}, x)
    # one panel; every row 5 long, so the sort moved no row (aux[3] = -1)
    assert h1.info()["aux"][3] == -1 and h1.info()["params"]["sell_panel_cols"] == a.n
    assert within_bound(a, x, y1)[0]


def test_padding_never_multiplied():
    """x[0] = NaN: padding slots hold column 0 but must never reach a product."""
    lens = np.array([1, 7, 2, 0, 30, 1, 3] * 40, np.int32)
    a = synth.from_lengths_random_cols(lens, 500, 3, "pad")
    a.idx[a.idx == 0] = 1
    x = synth.vector(a.n, 4)
    x[0] = np.nan
    for fmt in range(5):
        for p in PARAMS[fmt]:
            _, y = _run(a, fmt, p, x)
            assert np.all(np.isfinite(y)), (fmt, p)
            ok, msg = within_bound(a, x, y)
            assert ok, (fmt, p, msg)


def test_empty_matrix_gives_zero():
    a = synth.CSR(1000, 10, np.zeros(1001, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty")
    x = np.full(10, np.nan)
    for fmt in range(5):
        _, y = _run(a, fmt, None, x)
        assert np.all(y == 0.0) and not np.signbit(y).any(), fmt


# ------------------------------------------------------ layouts vs the oracle

def _np(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("mi", [1, 2, 5, 9])
def test_ell_layout_matches_oracle(mi):
    a = MATS[mi]
    h = sp.spmv_convert(sp.SPMV_ELL, sp.DeviceCSR.from_host(a))
    e = oracle.to_ell(a)
    K, m = e["K"], a.m
    ld = (m + 3) // 4 * 4
    assert h.info()["aux"][0] == K
    col = _np(h.array("col")).reshape(K, ld)[:, :m].reshape(-1)
    val = _np(h.array("val")).view(np.float64).reshape(K, ld)[:, :m].reshape(-1)
    assert np.array_equal(col, e["col"]) and np.array_equal(bits(val), bits(e["val"]))
    assert np.array_equal(_np(h.array("row_len"))[:m], e["row_len"])


@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 32), (64, 512), (128, -1), (32, 4096)])
@pytest.mark.parametrize("mi", [1, 2, 9])
def test_sell_layout_matches_oracle(C, sigma, mi):
    a = MATS[mi]
    h = sp.spmv_convert(sp.SPMV_SELL, sp.DeviceCSR.from_host(a), {"sell_C": C, "sell_sigma": sigma})
    s = oracle.to_sell(a, C, a.m if sigma == -1 or sigma > a.m else sigma)
    assert np.array_equal(_np(h.array("perm")), s["perm"])
    assert np.array_equal(_np(h.array("row_len"))[:a.m], s["row_len"])
    assert np.array_equal(_np(h.array("slice_ptr")), s["slice_ptr"])
    assert np.array_equal(_np(h.array("col")), s["col"])
    assert np.array_equal(bits(_np(h.array("val")).view(np.float64)), bits(s["val"]))
    # the product skips perm exactly when the oracle's order is the identity
    assert h.info()["aux"][3] == (-1 if np.array_equal(s["perm"], np.arange(a.m)) else 0)


@pytest.mark.parametrize("C,sigma", [(32, 1), (64, 1), (128, 1), (64, -1), (32, 64)])
def test_sell_identity_order_runs_without_perm(C, sigma):
    """Rows the sort leaves in place (sigma = 1, or equal lengths under any
    sigma): the handle reports it (aux[3] = -1) and the product, writing y
    without perm, matches the oracle; a matrix the sort reorders keeps perm."""
    m = 1000
    same = synth.uniform_random(m, 7, 3)  # every row 7 long: no sort moves a row
    mixed = synth.powerlaw(m, 11)
    for a, ident in ((same, True), (mixed, sigma == 1)):
        x = synth.vector(a.n, 5)
        h, y = _run(a, 3, {"sell_C": C, "sell_sigma": sigma}, x)
        s = oracle.to_sell(a, C, a.m if sigma == -1 else sigma)
        assert np.array_equal(s["perm"], np.arange(a.m)) == ident
        assert h.info()["aux"][3] == (-1 if ident else 0)
        ref = oracle.csr_spmv(a, x)
        assert np.all(np.abs(y - ref) <= oracle.fp_bound(a, x))


@pytest.mark.parametrize("mi", [1, 2, 3, 9])
def test_hyb_layout_matches_oracle(mi):
    a = MATS[mi]
    h = sp.spmv_convert(sp.SPMV_HYB, sp.DeviceCSR.from_host(a))
    o = oracle.to_hyb(a)
    K, m = o["K"], a.m
    assert h.info()["params"]["hyb_k"] == K
    ld = (m + 3) // 4 * 4
    col = _np(h.array("ell_col")).reshape(K, ld)[:, :m].reshape(-1)
    val = _np(h.array("ell_val")).view(np.float64).reshape(K, ld)[:, :m].reshape(-1)
    assert np.array_equal(col, o["col"]) and np.array_equal(bits(val), bits(o["val"]))
    rows, tptr = _np(h.array("tail_rows")), _np(h.array("tail_ptr"))
    ntr = len(tptr) - 1
    coo_row = np.repeat(rows[:ntr], np.diff(tptr))
    assert np.array_equal(coo_row, o["coo_row"])
    assert np.array_equal(_np(h.array("tail_col")), o["coo_col"])
    assert np.array_equal(bits(_np(h.array("tail_val")).view(np.float64)), bits(o["coo_val"]))


@pytest.mark.parametrize("sigma", [1, 3, 16, 32])
@pytest.mark.parametrize("mi", [0, 1, 2, 7, 9, 10])
def test_csr5_descriptors_match_oracle(sigma, mi):
    a = MATS[mi]
    h = sp.spmv_convert(sp.SPMV_CSR5, sp.DeviceCSR.from_host(a), {"csr5_sigma": sigma})
    o = oracle.to_csr5(a, 32, sigma)
    nt = o["ntiles"]
    assert h.info()["aux"][0] == nt
    assert np.array_equal(_np(h.array("tile_ptr")), o["tile_ptr"])
    words = _np(h.array("flags")).view(np.uint32).reshape(nt, 32)
    bitf = ((words[:, None, :] >> np.arange(sigma, dtype=np.uint32)[None, :, None]) & 1).astype(np.uint8)
    assert np.array_equal(bitf.reshape(-1), o["bit_flag"])  # slot (r, c) at r*32 + c
    assert np.array_equal(_np(h.array("y_off")), o["y_off"])
    seg = _np(h.array("seg_off")).view(np.uint32)
    segbits = ((seg[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1).astype(np.uint8).reshape(-1)
    assert np.array_equal(segbits, o["seg_off"])
    assert np.array_equal(_np(h.array("tile_idx")), o["idx"])
    assert np.array_equal(bits(_np(h.array("tile_val")).view(np.float64)), bits(o["val"]))
    assert np.array_equal(_np(h.array("empty_ptr")), o["empty_ptr"])
    assert np.array_equal(_np(h.array("empty_rows")), o["empty_rows"])


# ------------------------------------------------------------ error paths

def test_malformed_inputs_rejected():
    good = synth.powerlaw(1000, 5, xmax=50, lmax=50)
    bad_ptr = synth.CSR(good.m, good.n, good.ptr.copy(), good.idx, good.val)
    bad_ptr.ptr[10], bad_ptr.ptr[11] = bad_ptr.ptr[11], bad_ptr.ptr[10] + 1  # decreasing
    bad_idx = synth.CSR(good.m, good.n, good.ptr, good.idx.copy(), good.val)
    bad_idx.idx[5] = good.n
    for b in (bad_ptr, bad_idx):
        with pytest.raises(sp.SpmvError) as ei:
            sp.spmv_convert(sp.SPMV_CSR, sp.DeviceCSR.from_host(b))
        assert ei.value.name == "INVALID_ARG"


def test_too_large_and_alloc_failure():
    a = synth.powerlaw(20_000, 9, xmax=3000, lmax=3000)
    d = sp.DeviceCSR.from_host(a)
    with pytest.raises(sp.SpmvError) as ei:
        sp.spmv_convert(sp.SPMV_ELL, d, {"max_bytes": 1 << 20})
    assert ei.value.name == "TOO_LARGE"
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for fmt in range(5):
        for k in (1, 2, 4, 7):
            sp.spmv_debug_fail_alloc(k)
            try:
                sp.spmv_convert(fmt, d)
            except sp.SpmvError as e:
                assert e.name == "ALLOC"
            finally:
                sp.spmv_debug_fail_alloc(0)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)  # nothing leaked


def test_nnz_beyond_int32_refused():
    """nnz >= 2^31 does not fit the int32 row pointers: INDEX_OVERFLOW in every
    format, decided on the host before any of the CSR is read (the buffers
    behind this descriptor are a small valid matrix)."""
    a = synth.config1()
    d = sp.DeviceCSR.from_host(a)
    d._c = sp._abi.spmv_csr(a.m, a.n, 2**31, d.ptr.data_ptr(), d.idx.data_ptr(), d.val.data_ptr())
    for fmt in range(5):
        with pytest.raises(sp.SpmvError) as ei:
            sp.spmv_convert(fmt, d)
        assert ei.value.name == "INDEX_OVERFLOW", sp.FORMATS[fmt]
    d._c = sp._abi.spmv_csr(a.m, a.n, a.nnz, d.ptr.data_ptr(), d.idx.data_ptr(), d.val.data_ptr())
    sp.spmv_convert(0, d)  # the same buffers with their true nnz convert


def test_bad_arguments():
    a = synth.config1()
    d = sp.DeviceCSR.from_host(a)
    h = sp.spmv_convert(sp.SPMV_CSR, d)
    x = torch.zeros(a.n, dtype=torch.float64, device="cuda")
    with pytest.raises(sp.SpmvError):
        sp.spmv_run(h, x, x)  # aliasing
    with pytest.raises(sp.SpmvError):
        sp.spmv_convert(sp.SPMV_SELL, d, {"sell_C": 48})
    with pytest.raises(sp.SpmvError):
        sp.spmv_convert(sp.SPMV_CSR5, d, {"csr5_omega": 16})
    with pytest.raises(sp.SpmvError):
        sp.spmv_convert(sp.SPMV_CSR, d, {"csr_block_nnz": 1000})
    with pytest.raises(sp.SpmvError):
        sp.spmv_convert(sp.SPMV_CSR, d, {"csr_block_nnz": -3})


# --------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def cfg2():
    return synth.config2()


def test_full_size_ell_refused_under_cap(cfg2):
    d = sp.DeviceCSR.from_host(cfg2)
    with pytest.raises(sp.SpmvError) as ei:
        sp.spmv_convert(sp.SPMV_ELL, d, {"max_bytes": 8 << 30})
    assert ei.value.name == "TOO_LARGE"


def test_gather_probe_sums_every_product():
    """The benchmark's gather-ceiling probe touches every entry once: with integer values
    its partial sums add up exactly to sum(val[k] * x[idx[k]])."""
    for mi in (1, 9, 10):
        a = synth.with_integer_values(MATS[mi], 31 + mi)
        x = synth.integers(a.n, 32 + mi, -16, 16)
        part = probe.gather(sp.DeviceCSR.from_host(a), torch.as_tensor(x).cuda()).cpu().numpy()
        exact = int(np.sum(a.val.astype(np.int64) * x.astype(np.int64)[a.idx]))
        assert part.sum() == float(exact), (a.name, part.sum(), exact)
