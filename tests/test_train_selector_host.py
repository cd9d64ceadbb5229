"""Host-side pieces of the selector's training driver: the feature transform
it fits the scaling on (against the oracle's), the seeded split, and the
% of best measure with its fixed-format comparisons (closed forms)."""
import numpy as np
import pytest

from oracle import mlp
from paper_1805_11938_gb300 import train_selector as ts


def test_transform_matches_the_oracle():
    rng = np.random.default_rng(11)
    F = np.abs(rng.standard_normal((64, 16))) * 10.0 ** rng.integers(-3, 7, size=(64, 16))
    F[0] = 0.0          # empty matrix: every log argument at its floor
    F[1, 2] = 1e-30     # nnz fraction below the 2^-60 floor
    assert np.array_equal(ts.transform(F), mlp.transform(F))


def test_split_is_seeded_disjoint_and_complete():
    tr, te = ts.split(1000)
    tr2, te2 = ts.split(1000)
    assert np.array_equal(tr, tr2) and np.array_equal(te, te2)
    assert len(tr) == 800 and len(te) == 200
    assert not set(tr.tolist()) & set(te.tolist())
    assert sorted(tr.tolist() + te.tolist()) == list(range(1000))
    assert not np.array_equal(ts.split(1000, seed=1)[1], te)


def _records():
    # matrix 0: CSR 1 ms (best), SELL 2 ms; matrix 1: SELL 1 ms (best), CSR 4 ms, ELL infeasible
    base = {"CSR5": 8.0, "ELL": 8.0, "HYB": 8.0}
    return [{"ms": {**base, "CSR": 1.0, "SELL": 2.0}, "label": 0},
            {"ms": {**base, "CSR": 4.0, "SELL": 1.0, "ELL": None}, "label": 3}]


def test_pct_of_best_closed_forms():
    recs = _records()
    assert ts.pct_of_best(recs, [0, 1], [0, 3]).tolist() == [1.0, 1.0]
    assert ts.pct_of_best(recs, [0, 1], [3, 0]).tolist() == [0.5, 0.25]
    assert ts.pct_of_best(recs, [1], [2]).tolist() == [0.0]  # infeasible choice


def test_summary_fixed_formats_and_gains():
    s = ts.summary(_records(), [0, 1], [0, 3])
    assert s["mean_pct_of_best"] == pytest.approx(100.0) and s["accuracy"] == 1.0
    assert s["fixed_format_mean_pct_of_best"]["CSR"] == pytest.approx(100 * (1.0 + 0.25) / 2)
    assert s["fixed_format_mean_pct_of_best"]["SELL"] == pytest.approx(100 * (0.5 + 1.0) / 2)
    assert s["best_fixed_format"] == "SELL"
    assert s["gain_over_best_fixed_pct_points"] == pytest.approx(25.0)
    assert s["gain_over_always_csr_pct_points"] == pytest.approx(37.5)
    assert s["worst_pct_of_best"] == pytest.approx(100.0)
