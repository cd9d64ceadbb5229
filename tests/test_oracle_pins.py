"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Table I (the paper's worked example, tests/golden/table1.json), closed forms
(identity, permutation, diagonal, empty rows, the 5-point Laplacian), exact
integer arithmetic, numpy's dense product, exact rational sums, brute force on
tiny patterns, and finite differences for the selector network.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.json")


@pytest.fixture(scope="module")
def t1():
    with open(GOLDEN) as f:
        return json.load(f)


def table1_csr(t1):
    c = t1["csr"]
    return synth.CSR(t1["m"], t1["n"], np.array(c["ptr"], np.int32), np.array(c["indices"], np.int32),
                     np.array(c["data"], np.float64), "table1")


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def same_csr(a, ptr, idx, val):
    return (np.array_equal(a.ptr, ptr) and np.array_equal(a.idx, idx) and np.array_equal(bits(a.val), bits(val)))


# ------------------------------------------------------------------ Table I

def test_table1_coo_to_csr(t1):
    c = t1["coo"]
    ptr, idx, val = oracle.coo_to_csr(4, c["row"], c["col"], c["data"])
    assert ptr.tolist() == t1["csr"]["ptr"]
    assert idx.tolist() == t1["csr"]["indices"]
    assert val.tolist() == t1["csr"]["data"]


def test_table1_csr5(t1):
    g = t1["csr5"]
    t = oracle.to_csr5(table1_csr(t1), g["omega"], g["sigma"])
    assert t["ntiles"] == 2
    assert t["ptr"].tolist() == g["ptr"]
    assert t["tile_ptr"].tolist() == g["tile_ptr"]
    assert t["bit_flag"].astype(bool).tolist() == [b for tile in g["bit_flag"] for b in tile]
    assert t["y_off"].tolist() == [v for tile in g["y_off"] for v in tile]
    assert t["seg_off"].tolist() == [v for tile in g["seg_off"] for v in tile]
    assert t["idx"].tolist() == [v for tile in g["indices"] for v in tile]
    assert t["val"].tolist() == [v for tile in g["data"] for v in tile]
    assert t["empty_rows"].size == 0


def _ell_rows(col, val, row_len, m, K):
    """Row-major view of a column-major ELL, padding as None."""
    d = [[val[s * m + i] if s < row_len[i] else None for s in range(K)] for i in range(m)]
    c = [[int(col[s * m + i]) if s < row_len[i] else None for s in range(K)] for i in range(m)]
    return d, c


def test_table1_ell(t1):
    g = t1["ell"]
    e = oracle.to_ell(table1_csr(t1))
    assert e["K"] == g["K"]
    d, c = _ell_rows(e["col"], e["val"], e["row_len"], 4, e["K"])
    assert d == g["data"] and c == g["indices"]
    pad = np.array([[s >= e["row_len"][i] for i in range(4)] for s in range(3)]).reshape(-1)
    assert np.all(e["col"][pad] == 0) and np.all(bits(e["val"][pad]) == 0)  # +0.0 padding


@pytest.mark.parametrize("key", ["sell", "sell_c_sigma"])
def test_table1_sell(t1, key):
    g = t1[key]
    s = oracle.to_sell(table1_csr(t1), g["C"], g["sigma"])
    widths = (np.diff(s["slice_ptr"]) // g["C"]).tolist()
    assert widths == g["slices"]
    rows_d, rows_c = [], []
    for p in range(4):
        sl, l = divmod(p, g["C"])
        w = widths[sl]
        rows_d.append([s["val"][s["slice_ptr"][sl] + j * g["C"] + l] if j < s["row_len"][p] else None for j in range(w)])
        rows_c.append([int(s["col"][s["slice_ptr"][sl] + j * g["C"] + l]) if j < s["row_len"][p] else None for j in range(w)])
    assert rows_d == g["data"] and rows_c == g["indices"]
    if key == "sell_c_sigma":
        assert s["perm"].tolist() == [1, 0, 3, 2]
    else:
        assert s["perm"].tolist() == [0, 1, 2, 3]


def test_table1_hyb(t1):
    g = t1["hyb"]
    h = oracle.to_hyb(table1_csr(t1))
    assert h["K"] == g["K"]
    d, c = _ell_rows(h["col"], h["val"], h["row_len"], 4, h["K"])
    assert d == g["ell_data"] and c == g["ell_indices"]
    assert h["coo_row"].tolist() == g["coo"]["row"]
    assert h["coo_col"].tolist() == g["coo"]["col"]
    assert h["coo_val"].tolist() == g["coo"]["data"]


def test_table1_product(t1):
    """Table I's matrix times x = (1, 10, 100, 1000): each y_i read off the printed rows."""
    a = table1_csr(t1)
    y = oracle.csr_spmv(a, np.array([1.0, 10.0, 100.0, 1000.0]))
    assert y.tolist() == [6 * 10 + 1 * 100, 2 * 1 + 8 * 100 + 3 * 1000, 4 * 100, 7 * 10 + 5 * 100]


# -------------------------------------------------------------- closed forms

def diag_csr(d):
    n = len(d)
    return synth.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(d, np.float64))


def test_identity_gives_x():
    x = synth.vector(1000, 3)
    assert np.array_equal(bits(oracle.csr_spmv(diag_csr(np.ones(1000)), x)), bits(x))


def test_permutation_gives_permuted_x():
    n = 777
    pi = np.argsort(synth.vector(n, 11))
    a = synth.CSR(n, n, np.arange(n + 1, dtype=np.int32), pi.astype(np.int32), np.ones(n))
    x = synth.vector(n, 12)
    assert np.array_equal(bits(oracle.csr_spmv(a, x)), bits(x[pi]))


def test_diagonal_is_one_rounded_product():
    n = 500
    d = synth.vector(n, 21, -3, 3)
    x = synth.vector(n, 22)
    y = oracle.csr_spmv(diag_csr(d), x)
    assert np.array_equal(bits(y), bits(d * x))  # numpy's correctly rounded product


def test_empty_rows_are_positive_zero():
    a = synth.CSR(5, 3, np.array([0, 0, 2, 2, 3, 3], np.int32), np.array([0, 2, 1], np.int32), np.array([1.0, 2.0, 3.0]))
    x = np.array([np.inf, -5.0, np.nan])  # never touched by the empty rows
    y = oracle.csr_spmv(a, np.array([1.0, 1.0, 1.0]))
    assert y.tolist() == [0.0, 3.0, 0.0, 3.0, 0.0]
    assert not np.signbit(y[[0, 2, 4]]).any()
    y2 = oracle.csr_spmv(a, x)
    assert y2[0] == 0.0 and y2[2] == 0.0 and y2[4] == 0.0


@pytest.mark.parametrize("nx,ny", [(64, 64), (7, 3), (1, 5), (2, 2)])
def test_laplacian_rowsums(nx, ny):
    """5-point Laplacian times ones = 4 - (in-grid neighbours): 0 inside, 1 on edges, 2 at corners."""
    a = synth.laplacian2d(nx, ny)
    y = oracle.csr_spmv(a, np.ones(a.n))
    xs, ys = np.meshgrid(np.arange(nx), np.arange(ny))
    nb = (xs > 0).astype(int) + (xs < nx - 1) + (ys > 0) + (ys < ny - 1)
    assert y.tolist() == (4 - nb).reshape(-1).astype(float).tolist()


# ---------------------------------------------------------------- exactness

@pytest.mark.parametrize("seed", range(4))
def test_integer_valued_exact(seed):
    a = synth.with_integer_values(synth.powerlaw(3000, 100 + seed, xmax=300, lmax=300), seed)
    x = synth.integers(a.n, 50 + seed, -16, 16)
    y = oracle.csr_spmv(a, x)
    ptr, idx, val = a.ptr, a.idx, a.val.astype(np.int64)
    xi = x.astype(np.int64)
    exact = [int(sum(int(val[k]) * int(xi[idx[k]]) for k in range(ptr[i], ptr[i + 1]))) for i in range(a.m)]
    assert y.tolist() == [float(v) for v in exact]


def test_threads_bit_identical():
    a = synth.powerlaw(50_000, 5)
    x = synth.vector(a.n, 6)
    assert np.array_equal(bits(oracle.csr_spmv(a, x)), bits(oracle.csr_spmv_threads(a, x, 7)))


def _dense(a):
    d = np.zeros((a.m, a.n))
    for i in range(a.m):
        for k in range(a.ptr[i], a.ptr[i + 1]):
            d[i, a.idx[k]] += a.val[k]
    return d


@pytest.mark.parametrize("m,n,density,seed", [(1, 1, 1.0, 0), (8, 5, 0.4, 1), (64, 64, 0.1, 2), (33, 17, 0.6, 3),
                                              (10, 64, 0.0, 4), (5, 40, 1.0, 5)])
def test_against_numpy_dense(m, n, density, seed):
    a = synth.tiny_random(m, n, density, seed)
    x = synth.vector(n, seed + 99)
    y = oracle.csr_spmv(a, x)
    ref = _dense(a) @ x
    assert np.all(np.abs(y - ref) <= 2 * 4 * np.maximum(np.diff(a.ptr), 1) * 2.0 ** -53 * (np.abs(_dense(a)) @ np.abs(x)) + 0.0)
    yd = oracle.dense_matvec(_dense(a), x)
    assert np.all(np.abs(yd - ref) <= 2 * 4 * n * 2.0 ** -53 * (np.abs(_dense(a)) @ np.abs(x)))


def test_single_dense_row_and_empty_columns():
    d = np.zeros((3, 50))
    d[1, :] = synth.vector(50, 8)
    a = synth.from_dense(d)
    x = synth.vector(50, 9)
    y = oracle.csr_spmv(a, x)
    exact = sum(Fraction(float(d[1, j])) * Fraction(float(x[j])) for j in range(50))
    assert y[0] == 0.0 and y[2] == 0.0
    assert abs(Fraction(float(y[1])) - exact) <= Fraction(4 * 50) * Fraction(2.0 ** -53) * sum(abs(Fraction(float(d[1, j])) * Fraction(float(x[j]))) for j in range(50))


def test_within_error_bound_of_exact_sum():
    """The oracle's y is within 4*nnz_i*2^-53*sum|a x| of the exact rational row sums."""
    a = synth.powerlaw(400, 77, xmax=200, lmax=200)
    x = synth.vector(a.n, 78)
    y = oracle.csr_spmv(a, x)
    b = oracle.fp_bound(a, x)
    for i in range(a.m):
        ex = sum((Fraction(float(a.val[k])) * Fraction(float(x[a.idx[k]])) for k in range(a.ptr[i], a.ptr[i + 1])), Fraction(0))
        assert abs(Fraction(float(y[i])) - ex) <= Fraction(float(b[i]))



def test_fp_bound_hand_computed():
    """The tolerance 4 * nnz_i * 2^-53 * sum_j |a_ij x_j|, worked by hand row by
    row as exact multiples of 2^-53 (small integers and powers of two, so every
    step is exact in FP64).  Rows of different lengths catch a wrong nnz_i
    factor; signed entries catch a dropped absolute value; the duplicate pair
    cancels in y but not in the bound."""
    u = 2.0 ** -53
    # row 0: {2, -3} on x = (1, 1)             -> 4 * 2 * (2 + 3)       = 40 u
    # row 1: empty                              -> 0
    # row 2: {0.5} on x_1 = -4                  -> 4 * 1 * 2             =  8 u
    # row 3: {-2, 3, 1} on x = (-1, 2, -0.25)   -> 4 * 3 * (2 + 6 + 0.25) = 99 u
    # row 4: duplicates {1.5, -1.5} in column 0 -> 4 * 2 * (3 + 3)       = 48 u
    ptr = np.array([0, 2, 2, 3, 6, 8], np.int32)
    idx = np.array([0, 1, 1, 0, 1, 2, 0, 0], np.int32)
    val = np.array([2.0, -3.0, 0.5, -2.0, 3.0, 1.0, 1.5, -1.5])
    a = synth.CSR(5, 3, ptr, idx, val, "bound_rows")
    x = np.array([1.0, 1.0, 1.0])
    assert oracle.fp_bound(a, x)[[0, 1]].tolist() == [40 * u, 0.0]
    x = np.array([-1.0, -4.0, -0.25])
    b = oracle.fp_bound(a, x)
    assert b[1] == 0.0 and b[2] == 4 * 1 * 2.0 * u
    x = np.array([-1.0, 2.0, -0.25])
    b = oracle.fp_bound(a, x)
    assert b[3] == 4 * 3 * 8.25 * u
    x = np.array([2.0, 0.0, 0.0])
    b = oracle.fp_bound(a, x)
    assert b[4] == 48 * u and oracle.csr_spmv(a, x)[4] == 0.0
    assert b[0] == 4 * 2 * 4.0 * u  # |2 * 2| + |-3 * 0|
    # the bound scales with |x| and is zero exactly on rows whose products all vanish
    assert np.array_equal(oracle.fp_bound(a, 2.0 * x), 2.0 * b)
    assert oracle.fp_bound(a, np.zeros(3)).tolist() == [0.0] * 5


# ------------------------------------------------------- converters, brute force

def _patterns():
    """Small CSR patterns: empty rows, explicit zeros, -0.0, duplicates, unsorted columns."""
    out = []
    rng_seed = 0
    for m in range(1, 7):
        for trial in range(6):
            rng_seed += 1
            lens = [int(synth.u01(rng_seed, 1, i) * 5) for i in range(m)]
            if trial == 0:
                lens = [0] * m
            ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
            nnz = int(ptr[-1])
            idx = np.array([int(synth.u01(rng_seed, 2, k) * 4) for k in range(nnz)], np.int32)  # dup + unsorted
            val = synth.integers(nnz, rng_seed, -3, 3)
            if nnz > 1:
                val[0] = -0.0
            out.append(synth.CSR(m, 4, ptr, idx, val, f"p{m}_{trial}"))
    return out


PATTERNS = _patterns()


def test_roundtrip_ell_bruteforce():
    for a in PATTERNS:
        mx = oracle.max_row_len(a)
        for K in (mx, mx + 2):
            e = oracle.to_ell(a, K)
            assert same_csr(a, *oracle.ell_to_csr(a.m, e)), a.name


def test_roundtrip_sell_bruteforce():
    for a in PATTERNS:
        for C in (1, 2, 3, 4):
            for sigma in sorted({1, C, 2 * C, 4 * C, a.m}):
                s = oracle.to_sell(a, C, sigma)
                assert same_csr(a, *oracle.sell_to_csr(a.m, s)), (a.name, C, sigma)
                lens = np.diff(a.ptr)
                # window invariants: a permutation of the window, lengths non-increasing, ties in row order
                for b in range(0, a.m, sigma):
                    w = s["perm"][b:b + sigma]
                    assert sorted(w.tolist()) == list(range(b, min(b + sigma, a.m)))
                    key = [(-lens[r], r) for r in w]
                    assert key == sorted(key)
                assert np.array_equal(s["row_len"], lens[s["perm"]])
                widths = np.diff(s["slice_ptr"]) // C
                for sl in range(len(widths)):
                    assert widths[sl] == max(s["row_len"][sl * C:(sl + 1) * C].tolist() + [0])


def test_roundtrip_hyb_bruteforce():
    for a in PATTERNS:
        for K in range(0, oracle.max_row_len(a) + 2):
            h = oracle.to_hyb(a, K)
            assert same_csr(a, *oracle.hyb_to_csr(a.m, h)), (a.name, K)
            assert h["coo_row"].size == sum(max(0, l - K) for l in np.diff(a.ptr))


def _csr5_product(t, m, x):
    """y from the CSR5 arrays alone: walk each tile in nonzero order, start a new
    segment at every flagged slot, and send segment j of tile t to row
    tile_ptr[t] + j (or to the listed row for tiles with empty rows); a tile's
    first segment that continues a row adds to it."""
    om, sg = t["omega"], t["sigma"]
    S = om * sg
    y = [Fraction(0)] * m
    nnz = int(t["ptr"][-1])
    for tile in range(t["ntiles"]):
        base = tile * S
        listed = t["empty_rows"][t["empty_ptr"][tile]:t["empty_ptr"][tile + 1]].tolist()
        j = -1
        for c in range(om):
            assert t["y_off"][tile * om + c] == j + 1
            for r in range(sg):
                k = base + c * sg + r
                if k >= nnz:
                    break
                slot = base + r * om + c
                if t["bit_flag"][slot]:
                    j += 1
                row = listed[j] if listed else int(t["tile_ptr"][tile]) + j
                y[row] += Fraction(float(t["val"][slot])) * Fraction(float(x[t["idx"][slot]]))
    return y


def test_csr5_semantics_and_roundtrip_bruteforce():
    for a in PATTERNS:
        lens = np.diff(a.ptr)
        if a.nnz == 0:
            continue
        x = synth.integers(a.n, 5, -4, 4)
        ref = [sum((Fraction(float(a.val[k])) * Fraction(float(x[a.idx[k]])) for k in range(a.ptr[i], a.ptr[i + 1])), Fraction(0)) for i in range(a.m)]
        for om in (1, 2, 4):
            for sg in (1, 2, 3):
                t = oracle.to_csr5(a, om, sg)
                assert same_csr(a, *oracle.csr5_to_csr(a.m, a.nnz, t)), (a.name, om, sg)
                assert _csr5_product(t, a.m, x) == ref, (a.name, om, sg)
                assert t["tile_ptr"][-1] == a.m
                for tile in range(t["ntiles"]):
                    for c in range(om):
                        col = [t["bit_flag"][tile * om * sg + r * om + c] for r in range(sg)]
                        assert t["seg_off"][tile * om + c] == (sum(col) == 0)
        del lens


def test_csr5_empty_rows_listed():
    # rows: 0 -> 2 entries, 1 empty, 2 -> 1 entry, 3 empty, 4 -> 3 entries
    a = synth.CSR(5, 5, np.array([0, 2, 2, 3, 3, 6], np.int32), np.array([0, 1, 2, 3, 4, 0], np.int32),
                  np.arange(1.0, 7.0))
    t = oracle.to_csr5(a, 2, 2)  # tiles: nnz 0-3 (rows 0, 2, 4), nnz 4-5 (row 4)
    assert t["tile_ptr"].tolist() == [0, 4, 5]
    assert t["empty_ptr"].tolist() == [0, 3, 3]
    assert t["empty_rows"].tolist() == [0, 2, 4]


# ------------------------------------------------------------------- HYB rule

@pytest.mark.parametrize("lens,K", [([2, 3, 1, 2], 2), ([5, 5, 5, 5, 5], 5), ([0, 0, 7], 7), ([0, 0, 0, 0], 0),
                                    ([1, 2, 3, 4, 5, 6], 5), ([9], 9), ([1, 100, 1, 1, 1, 1], 1)])
def test_hyb_k_rule(lens, K):
    a = synth.CSR(len(lens), 200, np.concatenate([[0], np.cumsum(lens)]).astype(np.int32),
                  np.zeros(sum(lens), np.int32), np.ones(sum(lens)))
    assert oracle.hyb_k(a) == K
    assert oracle.hyb_k_of_lengths(lens) == K


# ------------------------------------------------------------------- features

def test_features_identity():
    f = oracle.features(diag_csr(np.ones(1000)))
    expect = [1000, 1000, 1e-3, 1, 1, 1, 0, 0, math.log2(1000), 1, 0, 0, 0, 0, 0, 1000 / (32 * 32)]
    assert np.allclose(f, expect, rtol=1e-15, atol=0)


def test_features_laplacian_64():
    """Counted by hand: 4 corner rows of 3 entries, 248 edge rows of 4, 3844 interior rows of 5."""
    f = oracle.features(synth.laplacian2d(64, 64))
    n, nnz = 4096, 4 * 3 + 248 * 4 + 3844 * 5
    mean = nnz / n
    var = (4 * 9 + 248 * 16 + 3844 * 25) / n - mean ** 2
    # |col - row| per entry: 0 (diagonal), 1 per x-neighbour, 64 per y-neighbour
    x_nb = 2 * 63 * 64  # 63 left and 63 right neighbours on each of 64 grid lines
    y_nb = 2 * 63 * 64
    assert n + x_nb + y_nb == nnz
    spread = (1 * x_nb + 64 * y_nb) / nnz
    sell_denom = 32 * (3 * 128 + 128 + 121)  # c_1..c_3 = 4096, c_4 = 4092, c_5 = 3844
    expect = [n, n, nnz / n ** 2, 3, 5, mean, math.sqrt(var), math.sqrt(var) / mean, math.log2(nnz), mean / 5, 0.0,
              spread, 64, 0, 0, nnz / sell_denom]
    assert np.allclose(f, expect, rtol=1e-12, atol=1e-15)


def test_features_sampled_rows():
    """Above 8192 rows the row-length statistics stay exact over all rows,
    while the histogram features (10, 15) and the index spread (11, 12) see only
    rows floor(k*M/8192).  Here exactly the sampled rows are long (40 entries)
    and every other row is empty; the values are counted by hand."""
    m = 40_000
    sampled = set((k * m) // 8192 for k in range(8192))
    assert len(sampled) == 8192
    lens = np.array([40 if i in sampled else 0 for i in range(m)], np.int32)
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    idx = np.concatenate([np.arange(40) for _ in sampled]).astype(np.int32)
    a = synth.CSR(m, 40, ptr, idx, np.ones(int(ptr[-1])))
    f = oracle.features(a)
    nnz = 40 * 8192
    assert f[3] == 0 and f[4] == 40  # exact: the empty rows count
    assert f[5] == nnz / m
    # population std over all rows: sqrt(M * 8192 * 40^2 - nnz^2) / M
    assert f[6] == math.sqrt(m * 8192 * 1600 - nnz * nnz) / m
    assert f[7] == f[6] / (nnz / m) and f[9] == (nnz / m) / 40
    assert f[13] == (m - 8192) / m and f[14] == 8192 / m
    # the sample sees only rows of 40: K = 40, no tail; SELL-32 slices all full
    assert f[10] == 0.0 and f[15] == 1.0


def test_features_long_row_the_sample_misses():
    """Rows of one entry and a single row of 5000 entries at row 1, which the
    row sample (rows floor(k*40000/8192): 0, 4, 9, ...) skips: the exact
    statistics see it, the sampled features do not."""
    m = 40_000
    assert 1 not in set((k * m) // 8192 for k in range(8192))
    lens = np.ones(m, np.int32)
    lens[1] = 5000
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    idx = np.concatenate([np.array([i % 7000]) if i != 1 else np.arange(5000) for i in range(m)]).astype(np.int32)
    a = synth.CSR(m, 7000, ptr, idx, np.ones(int(ptr[-1])))
    f = oracle.features(a)
    nnz = m - 1 + 5000
    assert f[4] == 5000 and f[3] == 1 and f[5] == nnz / m
    assert f[6] == math.sqrt(m * (m - 1 + 5000 ** 2) - nnz * nnz) / m
    assert f[9] == (nnz / m) / 5000 and f[14] == 1 / m and f[13] == 0
    assert f[10] == 0.0 and f[15] == 1.0  # sampled: all of length 1, K = 1, full slices


def test_features_empty_and_long():
    lens = [0, 0, 0, 40, 1, 1]
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    a = synth.CSR(6, 100, ptr, np.arange(int(ptr[-1]), dtype=np.int32) % 100, np.ones(int(ptr[-1])))
    f = oracle.features(a)
    assert f[13] == 0.5 and f[14] == 1 / 6
    assert oracle.hyb_k_of_lengths(lens) == 1  # ceil(6/3) = 2 rows with >= 1
    assert f[10] == 39 / 42
    # SELL-32 over 6 rows: one slice, width 40 -> fill 42 / (32 * 40)
    assert f[15] == 42 / (32 * 40)


# ---------------------------------------------------------------------- MLP

def _theta(seed):
    return mlp.glorot_init(synth.vector(mlp.N_PARAMS, seed))


def test_mlp_param_count():
    assert mlp.N_PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 64 * 5 + 5 == 5573


def test_mlp_zero_weights_closed_form():
    x = synth.vector(10 * 16, 3, 0, 1).reshape(10, 16)
    labels = np.array([0, 1, 2, 3, 4, 0, 0, 1, 1, 4])
    loss, g = mlp.loss_and_grad(np.zeros(mlp.N_PARAMS), x, labels)
    assert loss == pytest.approx(math.log(5), rel=1e-15)
    gp = mlp.unpack(g)
    freq = np.bincount(labels, minlength=5) / 10
    assert np.allclose(gp["b3"], 0.2 - freq, atol=1e-16)
    for name in ("W1", "b1", "W2", "b2", "W3"):
        assert not np.any(gp[name])


def test_mlp_forward_hand_example():
    """W1 copies the first 3 inputs, W2 is the identity, W3 sums them into class 2."""
    p = {n: np.zeros(s) for n, s in mlp.SHAPES}
    p["W1"][0, 0] = p["W1"][1, 1] = p["W1"][2, 2] = 1.0
    p["b1"][3] = -1.0  # negative pre-activation: ReLU must cut it
    p["W1"][0, 3] = 0.5
    p["W2"] = np.eye(64)
    p["W3"][0:4, 2] = 1.0
    p["b3"][4] = 0.25
    x = np.zeros((1, 16))
    x[0, :3] = [0.5, 0.25, 0.125]
    z, _ = mlp.forward(mlp.pack(p), x)
    assert z.tolist() == [[0.0, 0.0, 0.875, 0.0, 0.25]]
    assert mlp.predict(mlp.pack(p), x).tolist() == [2]


@pytest.mark.parametrize("seed", [1, 2])
def test_mlp_gradient_finite_differences(seed):
    theta = _theta(seed)
    x = synth.vector(12 * 16, seed + 10, 0, 1).reshape(12, 16)
    labels = (np.arange(12) * 7 + seed) % 5
    _, g = mlp.loss_and_grad(theta, x, labels)
    h = 1e-6
    picks = [int(synth.u01(seed, 3, k) * mlp.N_PARAMS) for k in range(60)] + [0, 5572, 1024, 1088, 5568]
    for j in picks:
        e = np.zeros_like(theta)
        e[j] = h
        fd = (mlp.loss(theta + e, x, labels) - mlp.loss(theta - e, x, labels)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1e-3, abs(g[j])) + 1e-9, j


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -2.0, 1e-3, 0.0])
    th, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=0.0 + 1e-12)
    assert np.allclose(th[:3], [-0.01, 0.01, -0.01], rtol=1e-9)
    assert th[3] == 0.0
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)



def test_adam_constant_gradient_moves_lr_every_step():
    """With a constant gradient g, Adam's bias-corrected moments are exactly g
    and g^2 at every step t (m_t = (1 - beta1^t) g, v_t = (1 - beta2^t) g^2),
    so each step moves every parameter by lr against the sign of g.  A wrong
    step number in the bias correction breaks this from t = 2 on (with t = 1
    throughout, step 2 would move by lr * 1.9 / sqrt(1.999))."""
    g = np.array([3.0, -2.0, 1e-3, 0.5])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 6):
        prev = th
        th, m, v = mlp.adam_step(th, g, m, v, t, lr=0.01, eps=0.0)
        assert np.allclose(prev - th, 0.01 * np.sign(g), rtol=1e-9, atol=0), t


def test_adam_steps_two_and_three_hand_worked():
    """Gradient 1 at step 1, then 0 at steps 2 and 3 (beta1 0.9, beta2 0.999,
    lr 0.01).  By hand: m_2 = 0.09, v_2 = 0.000999, so the step-2 move is
    0.01 * (0.09 / 0.19) / sqrt(0.000999 / 0.001999) = 0.01 * (9/19) /
    sqrt(999/1999); m_3 = 0.081, v_3 = 0.000998001, and the step-3 move is
    0.01 * (81/271) / sqrt(998001/2997001)."""
    th, m, v = mlp.adam_step(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1, lr=0.01, eps=0.0)
    assert th[0] == pytest.approx(-0.01, rel=1e-12)
    th2, m, v = mlp.adam_step(th, np.zeros(1), m, v, 2, lr=0.01, eps=0.0)
    assert m[0] == pytest.approx(0.09, rel=1e-14) and v[0] == pytest.approx(0.000999, rel=1e-14)
    assert th[0] - th2[0] == pytest.approx(0.01 * (9 / 19) / math.sqrt(999 / 1999), rel=1e-12)
    th3, m, v = mlp.adam_step(th2, np.zeros(1), m, v, 3, lr=0.01, eps=0.0)
    assert m[0] == pytest.approx(0.081, rel=1e-14) and v[0] == pytest.approx(0.000998001, rel=1e-14)
    assert th2[0] - th3[0] == pytest.approx(0.01 * (81 / 271) / math.sqrt(998001 / 2997001), rel=1e-12)


def test_scaling_min_max():
    t = np.array([[1.0, 5.0, 2.0], [3.0, 5.0, 4.0], [2.0, 5.0, 0.0]])
    lo, hi = mlp.fit_scaling(t)
    x = mlp.scale(np.array([[2.0, 5.0, 8.0], [0.0, 1.0, 1.0]]), lo, hi)
    assert x.tolist() == [[0.5, 0.0, 1.0], [0.0, 0.0, 0.25]]


def test_transform():
    f = np.zeros(16)
    f[0] = 7.0
    f[2] = 2.0 ** -10
    f[7] = 0.3
    t = mlp.transform(f)
    assert t[0] == 3.0 and t[2] == 10.0 and t[7] == 0.3 and t[1] == 0.0
