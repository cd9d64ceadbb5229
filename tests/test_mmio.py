"""Matrix Market reading (CPU): hand-written files against their dense matrices."""
import gzip

import numpy as np
import pytest

import oracle
from paper_1805_11938_gb300.mmio import read_mtx


def _dense(a):
    d = np.zeros((a.m, a.n))
    for i in range(a.m):
        for k in range(a.ptr[i], a.ptr[i + 1]):
            d[i, a.idx[k]] += a.val[k]
    return d


def test_general_real_with_duplicates_and_comments(tmp_path):
    p = tmp_path / "g.mtx"
    p.write_text("%%MatrixMarket matrix coordinate real general\n% a comment\n\n3 4 5\n"
                 "1 2 1.5\n3 1 -2\n1 4 4e0\n1 2 0.5\n2 3 7\n")
    a = read_mtx(p)
    assert (a.m, a.n, a.nnz) == (3, 4, 5)
    assert a.ptr.tolist() == [0, 3, 4, 5]
    assert a.idx.tolist() == [1, 3, 1, 2, 0]  # file order inside row 0, the duplicate kept
    ref = np.array([[0, 2.0, 0, 4.0], [0, 0, 7.0, 0], [-2.0, 0, 0, 0]])
    assert np.array_equal(_dense(a), ref)
    x = np.array([1.0, 2.0, 3.0, 4.0])
    assert np.array_equal(oracle.csr_spmv(a, x), ref @ x)


def test_symmetric_pattern_and_skew(tmp_path):
    p = tmp_path / "s.mtx"
    p.write_text("%%MatrixMarket matrix coordinate pattern symmetric\n3 3 3\n1 1\n2 1\n3 2\n")
    a = read_mtx(p)
    assert np.array_equal(_dense(a), np.array([[1.0, 1, 0], [1, 0, 1], [0, 1, 0]]))
    q = tmp_path / "k.mtx.gz"
    with gzip.open(q, "wt") as f:
        f.write("%%MatrixMarket matrix coordinate integer skew-symmetric\n3 3 2\n2 1 5\n3 1 -2\n")
    b = read_mtx(q)
    assert np.array_equal(_dense(b), np.array([[0.0, -5, 2], [5, 0, 0], [-2, 0, 0]]))


def test_refuses_what_it_cannot_read(tmp_path):
    for text in ("%%MatrixMarket matrix array real general\n2 2\n1\n2\n3\n4\n",
                 "%%MatrixMarket matrix coordinate complex general\n1 1 1\n1 1 1 0\n",
                 "%%MatrixMarket matrix coordinate real general\n2 2 1\n3 1 1.0\n",
                 "not a matrix\n"):
        p = tmp_path / "bad.mtx"
        p.write_text(text)
        with pytest.raises(ValueError):
            read_mtx(p)
