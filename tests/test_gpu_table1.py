"""The paper's worked example (Sec. II-B, Table I) through the GPU path.

The 4 x 4 matrix of Table I is converted on the device through the C ABI and
each layout is read back and compared with the printed arrays
(tests/golden/table1.json): ELL (stored column-major here, the printed rows
read off it), SELL-C-sigma with the whole matrix as the sorting window (the
printed row order [1, 0, 3, 2] and rows; slices of C = 32 rows on the GPU
instead of the printed C = 2), plain SELL (sigma = 1), and HYB with the K
the typical-length rule gives (K = 2, the COO tail (1, 3, 3)).  CSR5 runs
with the GPU's tile width of 32, so only its product and way back are
compared.  Every format's product with x = (1, 10, 100, 1000) is the one
read off the printed rows, bit for bit, and every way back is exact.
"""
import json
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.json")


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


@pytest.fixture(scope="module")
def t1():
    with open(GOLDEN) as f:
        return json.load(f)


def _csr(t1):
    c = t1["csr"]
    return synth.CSR(4, 4, np.array(c["ptr"], np.int32), np.array(c["indices"], np.int32),
                     np.array(c["data"], np.float64), "table1")


def _arr(h, name, dtype=None):
    a = h.array(name).cpu().numpy()
    return a.view(dtype) if dtype is not None else a


def _rows(col, val, row_len, ld, width, order=range(4)):
    """Row-major view of a column-major layout (slot s of row/position p at s*ld + p), padding as None."""
    d = [[float(val[s * ld + p]) if s < row_len[p] else None for s in range(width)] for p in order]
    c = [[int(col[s * ld + p]) if s < row_len[p] else None for s in range(width)] for p in order]
    return d, c


def _trim(rows):
    return [r[:max([i + 1 for i, v in enumerate(r) if v is not None] or [0])] for r in rows]


def test_table1_products_and_round_trips(sp, t1):
    a = _csr(t1)
    d = sp.DeviceCSR.from_host(a)
    x = torch.tensor([1.0, 10.0, 100.0, 1000.0], dtype=torch.float64, device="cuda")
    expect = [6 * 10 + 1 * 100, 2 * 1 + 8 * 100 + 3 * 1000, 4 * 100, 7 * 10 + 5 * 100]
    for fmt in range(5):
        for params in (None, {"sell_sigma": 1}, {"sell_C": 128}) if fmt == 3 else (None,):
            h = sp.spmv_convert(fmt, d, params)
            assert sp.spmv_run(h, x).cpu().numpy().tolist() == expect, (fmt, params)
            p, i, v = (t.cpu().numpy() for t in sp.spmv_to_csr(h))
            assert p.tolist() == t1["csr"]["ptr"] and i.tolist() == t1["csr"]["indices"], fmt
            assert v.tolist() == t1["csr"]["data"], fmt


def test_table1_ell_layout(sp, t1):
    h = sp.spmv_convert(sp.SPMV_ELL, sp.DeviceCSR.from_host(_csr(t1)))
    g = t1["ell"]
    info = h.info()
    assert info["aux"][0] == g["K"]
    row_len = _arr(h, "row_len")
    d, c = _rows(_arr(h, "col"), _arr(h, "val", np.float64), row_len, 4, g["K"])
    assert d == g["data"] and c == g["indices"]


@pytest.mark.parametrize("key,params", [("sell_c_sigma", {"sell_sigma": -1}), ("sell", {"sell_sigma": 1})])
def test_table1_sell_layout(sp, t1, key, params):
    h = sp.spmv_convert(sp.SPMV_SELL, sp.DeviceCSR.from_host(_csr(t1)), params)
    g = t1[key]
    perm = _arr(h, "perm")
    assert perm.tolist() == ([1, 0, 3, 2] if key == "sell_c_sigma" else [0, 1, 2, 3])
    row_len = _arr(h, "row_len")  # per sorted position, padded to one slice of 32
    slice_ptr = _arr(h, "slice_ptr")
    assert slice_ptr.tolist() == [0, 32 * 3]  # one slice of C = 32 rows, three slots wide
    d, c = _rows(_arr(h, "col"), _arr(h, "val", np.float64), row_len, 32, 3)
    # the printed rows (slices of C = 2 trim each slice to its own width)
    assert _trim(d) == _trim(g["data"]) and _trim(c) == _trim(g["indices"])


def test_table1_hyb_layout(sp, t1):
    h = sp.spmv_convert(sp.SPMV_HYB, sp.DeviceCSR.from_host(_csr(t1)))
    g = t1["hyb"]
    info = h.info()
    assert info["params"]["hyb_k"] == g["K"] and info["aux"][0] == 1  # K = 2, one COO entry
    d, c = _rows(_arr(h, "ell_col"), _arr(h, "ell_val", np.float64), _arr(h, "ell_row_len"), 4, g["K"])
    assert d == g["ell_data"] and c == g["ell_indices"]
    ntr = info["aux"][1]  # rows with a tail (the row array has one entry more)
    assert ntr == 1 and _arr(h, "tail_rows")[:ntr].tolist() == g["coo"]["row"]
    assert _arr(h, "tail_ptr").tolist() == [0, 1]
    assert _arr(h, "tail_col").tolist() == g["coo"]["col"]
    assert _arr(h, "tail_val", np.float64).tolist() == g["coo"]["data"]
