"""What the trained selectors gain over the method without them (CPU).

Uses the committed profiling table (every corpus matrix timed in all five
formats on the GB300 by the library itself) and the committed networks.  The
oracle's FP64 network predicts the held-out matrices from their stored
features; the result is scored with the paper's measure (Sec. V-C):
performance of the predicted format relative to the exhaustively best one.
Without the network the choice is one fixed format for every matrix
(Table III's setting) or always CSR.

Two models are checked against their own timings: selector_mlp.json against
"ms" (one product of the matrix alone) and selector_mlp_batch.json against
"ms_batch" (throughput per copy of a block-diagonal replica, the regime of the
batched kernel).
"""
import json
import os

import numpy as np
import pytest

from oracle import mlp

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1805_11938_gb300", "data")
FORMATS = ("CSR", "CSR5", "ELL", "SELL", "HYB")


@pytest.fixture(scope="module")
def table():
    with open(os.path.join(DATA, "corpus_table.jsonl")) as f:
        recs = sorted((json.loads(l) for l in f), key=lambda r: r["index"])
    assert [r["index"] for r in recs] == list(range(len(recs)))
    return recs


MODELS = {"ms": "selector_mlp.json", "ms_batch": "selector_mlp_batch.json"}
# required gain over the best single format: in the throughput regime the best
# fixed format (HYB) is already within about 7 % of the exhaustive best, which
# bounds any selector's gain there
MARGIN = {"ms": 0.10, "ms_batch": 0.03}
LABEL = {"ms": "label", "ms_batch": "label_batch"}
BEST = {"ms": "best", "ms_batch": "best_batch"}


def _model(key):
    with open(os.path.join(DATA, MODELS[key])) as f:
        return json.load(f)


def _split(n):
    import synth

    keys = np.array([synth.u01(0, 0x5B117, i) for i in range(n)])
    order = np.argsort(keys, kind="stable")
    return np.sort(order[:800]), np.sort(order[800:])


def _pct(recs, idx, choice, key="ms"):
    out = []
    for i, c in zip(idx, choice):
        best = min(v for v in recs[i][key].values() if v is not None)
        t = recs[i][key][FORMATS[int(c)]]
        out.append(0.0 if t is None else best / t)
    return np.array(out)


def _predict(model, F):
    t = mlp.transform(F.astype(np.float32).astype(np.float64))
    x = mlp.scale(t, np.array(model["lo"], np.float64), np.array(model["hi"], np.float64))
    return mlp.predict(np.array(model["params"], np.float64), x)


@pytest.mark.parametrize("key", sorted(MODELS))
def test_table_labels_are_the_fastest_format(table, key):
    for r in table:
        feas = {k: v for k, v in r[key].items() if v is not None}
        assert r[BEST[key]] == min(feas, key=feas.get) and FORMATS[r[LABEL[key]]] == r[BEST[key]]
        assert len(r["features"]) == 16
        if r["replicas"] == 1:
            assert r["ms_batch"] == r["ms"]  # no replica: the throughput time is the single-product time


@pytest.mark.parametrize("key", sorted(MODELS))
def test_scaling_table_is_training_minmax(table, key):
    model = _model(key)
    assert model["timing"] == key
    tr, _ = _split(len(table))
    t = mlp.transform(np.array([table[i]["features"] for i in tr], np.float64))
    assert np.allclose(model["lo"], t.min(axis=0), rtol=1e-6, atol=1e-6)
    assert np.allclose(model["hi"], t.max(axis=0), rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("key", sorted(MODELS))
def test_selector_beats_every_fixed_format_on_held_out(table, key):
    model = _model(key)
    _, te = _split(len(table))
    F = np.array([table[i]["features"] for i in te])
    pred = _predict(model, F)
    mine = _pct(table, te, pred, key)
    fixed = {f: _pct(table, te, [k] * len(te), key).mean() for k, f in enumerate(FORMATS)}
    best_fixed = max(fixed.values())
    assert mine.mean() >= 0.95  # the 95%-of-best target
    assert mine.mean() >= best_fixed + MARGIN[key]  # over the best single format
    assert mine.mean() >= fixed["CSR"] + 0.10  # and over "always CSR"
    # the stored evaluation (made on the GPU by the library's kernels) agrees with the oracle's
    assert abs(100 * mine.mean() - model["held_out"]["mean_pct_of_best"]) < 1.0
