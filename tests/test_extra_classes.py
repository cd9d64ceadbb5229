"""The seven-class evaluation (plain SELL and COO beside the paper's five) on a
synthetic table whose answers are known in closed form."""
import numpy as np
import pytest

from paper_1805_11938_gb300 import extra_classes as ec
from paper_1805_11938_gb300.train_selector import split

NAMES = list(ec.BASE) + ["SELL_plain", "COO"]


def test_best_and_pct():
    ms = {"CSR": 3.0, "CSR5": 2.0, "ELL": None, "SELL": 4.0, "HYB": 5.0, "SELL_plain": 1.0, "COO": 6.0}
    assert ec.best(ms, ec.BASE) == ("CSR5", 2.0)
    assert ec.best(ms, NAMES) == ("SELL_plain", 1.0)
    assert ec.pct_vs(ms, NAMES, "CSR") == pytest.approx(1.0 / 3.0)
    assert ec.pct_vs(ms, NAMES, "ELL") == 0.0  # infeasible


def _table(n=60):
    """Feature 3 (min row length) decides: below 10 plain SELL is fastest (1 ms) and
    SELL the best of the five (2 ms); otherwise CSR (1 ms), everything else 3 ms."""
    recs = []
    for i in range(n):
        small = i % 3 == 0
        f = [1000.0 + i, 1000.0, 1e-3, 2.0 if small else 20.0, 50.0, 8.0] + [1.0] * 10
        if small:
            ms = {"CSR": 3.0, "CSR5": 3.0, "ELL": 3.0, "SELL": 2.0, "HYB": 3.0, "SELL_plain": 1.0, "COO": 3.0}
        else:
            ms = {"CSR": 1.0, "CSR5": 3.0, "ELL": 3.0, "SELL": 3.0, "HYB": 3.0, "SELL_plain": 3.0, "COO": 3.0}
        recs.append({"index": i, "classes": NAMES, "features": f, "ms": ms, "ms_batch": ms})
    return recs


def test_evaluate_closed_forms():
    recs = _table()
    r = ec.evaluate(recs, "ms")
    frac = np.mean([i % 3 == 0 for i in range(60)])
    assert r["best_counts"]["SELL_plain"] == 20 and r["best_counts"]["CSR"] == 40
    assert r["extra_best_fraction"] == pytest.approx(frac)
    # best of seven is 2x faster on the small-row matrices, equal elsewhere
    assert r["oracle_speedup_of_best7_over_best5"]["mean"] == pytest.approx(2 * frac + (1 - frac))
    assert r["oracle_speedup_of_best7_over_best5"]["max"] == pytest.approx(2.0)
    assert r["best5_pct_of_best7_mean"] == pytest.approx(100 * (0.5 * frac + (1 - frac)))
    # a separable feature: the seven-class tree is exact, the five-class one reaches the five-class optimum
    _, te = split(60, n_train=48)
    small_te = np.mean([i % 3 == 0 for i in te])
    assert r["seven_classes"]["DTC (the paper's)"]["mean_pct_of_best7"] == pytest.approx(100.0)
    assert r["five_classes"]["DTC (the paper's)"]["mean_pct_of_best7"] == pytest.approx(
        100 * (0.5 * small_te + (1 - small_te)))
    assert r["held_out_best5_pct_of_best7"] == pytest.approx(100 * (0.5 * small_te + (1 - small_te)))


def test_profiler_class_lists():
    """The five classes are the library's formats in id order (the labels of the shipped
    tables); the two extra ones are settings of existing kernels."""
    from paper_1805_11938_gb300 import FORMATS, SPMV_HYB_K_NONE, profile_corpus as pc

    assert [c[0] for c in pc.CLASSES_5] == list(FORMATS)
    assert [c[1] for c in pc.CLASSES_5] == list(range(5))
    assert all(c[2] == {} for c in pc.CLASSES_5)
    extra = {c[0]: c for c in pc.CLASSES_7[5:]}
    assert pc.CLASSES_7[:5] == pc.CLASSES_5
    assert extra["SELL_plain"][1] == 3 and extra["SELL_plain"][2] == {"sell_sigma": 1}
    assert extra["COO"][1] == 4 and extra["COO"][2] == {"hyb_k": SPMV_HYB_K_NONE}
    assert [c[0] for c in pc.CLASSES_7] == NAMES


def test_committed_results_reproduce():
    """data/selector_seven_classes.json is what extra_classes computes from the committed
    seven-class table."""
    import json
    import os

    from paper_1805_11938_gb300.train_selector import load_table

    data = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1805_11938_gb300", "data")
    recs = load_table(os.path.join(data, "corpus_table7.jsonl"))
    with open(os.path.join(data, "selector_seven_classes.json")) as f:
        stored = json.load(f)
    got = json.loads(json.dumps({key: ec.evaluate(recs, key) for key in ("ms", "ms_batch")}))
    assert got == stored


def test_replica_is_block_diagonal():
    """The throughput label's matrix diag(A, ..., A): k copies of A's rows, columns
    shifted by the copy, values repeated; its product is k copies of A x."""
    import synth
    import oracle
    from paper_1805_11938_gb300 import profile_corpus as pc

    a = synth.tiny_random(7, 5, 0.5, 21)
    r = pc.replica(a, 3)
    assert (r.m, r.n, int(r.ptr[-1])) == (3 * a.m, 3 * a.n, 3 * a.nnz)
    x = synth.vector(r.n, 4)
    y = oracle.csr_spmv(r, x)
    for c in range(3):
        assert np.array_equal(y[c * a.m:(c + 1) * a.m], oracle.csr_spmv(a, x[c * a.n:(c + 1) * a.n]))
    assert pc.replica(a, 1) is a


def test_replica_count_rule():
    """About 2^23 nonzeros in the replica, one copy for large or empty matrices, indices within int32."""
    import synth
    from paper_1805_11938_gb300 import profile_corpus as pc

    a = synth.tiny_random(7, 5, 0.5, 21)
    k = pc.replica_count(a)
    assert k * a.nnz >= pc.REPLICA_NNZ and (k - 1) * a.nnz < pc.REPLICA_NNZ
    assert k * max(a.m, a.n) < 2**31
    empty = synth.from_lengths_random_cols(np.zeros(4, np.int32), 3, 1, "empty")
    assert pc.replica_count(empty) == 1
