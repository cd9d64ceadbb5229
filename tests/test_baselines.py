"""The paper's decision tree and the alternatives of Sec. V-D (CPU), pinned to
their definitions: brute-force split search, the pure-leaf property of a fully
grown tree, and scikit-learn's routines where they exist (not on every box)."""
import json
import os

import numpy as np
import pytest

from paper_1805_11938_gb300 import baselines as bl

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1805_11938_gb300", "data")


def _data(seed, n=60, d=4, classes=5, distinct=True):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 7, size=(n, d)).astype(np.float64) if not distinct else rng.normal(size=(n, d))
    y = rng.integers(0, classes, size=n)
    return X, y


def _gini_counts(labels, classes=5):
    if len(labels) == 0:
        return 0.0
    p = np.bincount(labels, minlength=classes) / len(labels)
    return 1.0 - float((p * p).sum())


@pytest.mark.parametrize("seed", range(6))
def test_best_split_is_the_brute_force_optimum(seed):
    """Every feature and every midpoint between distinct values, impurity computed
    with plain loops: the search returns the minimum (first in feature, then
    threshold order)."""
    X, y = _data(seed, n=25, d=3, distinct=(seed % 2 == 0))
    best = None
    for j in range(X.shape[1]):
        vals = sorted(set(X[:, j]))
        for a, b in zip(vals[:-1], vals[1:]):
            t = 0.5 * (a + b)
            left, right = y[X[:, j] <= t], y[X[:, j] > t]
            imp = (len(left) * _gini_counts(left) + len(right) * _gini_counts(right)) / len(y)
            if best is None or imp < best[2] - 1e-15:
                best = (j, t, imp)
    got = bl.best_split(X, y)
    assert got[0] == best[0] and got[1] == best[1] and abs(got[2] - best[2]) < 1e-12


def test_fully_grown_tree_fits_distinct_training_points():
    X, y = _data(7, n=200, d=5)
    t = bl.DecisionTree().fit(X, y)
    assert np.array_equal(t.predict(X), y)  # pure leaves: every training sample classified
    stump = bl.DecisionTree(max_depth=1).fit(X, y)
    assert stump.depth() == 1 and len(stump.nodes) == 3


def test_tree_stump_impurity_matches_sklearn():
    sk = pytest.importorskip("sklearn.tree")
    X, y = _data(8, n=120, d=6)
    j, t, imp = bl.best_split(X, y)
    ref = sk.DecisionTreeClassifier(max_depth=1, random_state=0).fit(X, y).tree_
    n_l, n_r = ref.n_node_samples[1], ref.n_node_samples[2]
    ref_imp = (n_l * ref.impurity[1] + n_r * ref.impurity[2]) / len(y)
    assert abs(imp - ref_imp) < 1e-12  # the optimum is unique in value, whatever feature wins a tie


def test_gaussian_nb_matches_sklearn():
    nb = pytest.importorskip("sklearn.naive_bayes")
    X, y = _data(9, n=300, d=6)
    Xt, _ = _data(10, n=100, d=6)
    ours = bl.GaussianNB().fit(X, y)
    ref = nb.GaussianNB().fit(X, y)
    assert np.array_equal(ours.predict(Xt), ref.predict(Xt))
    assert np.allclose(ours.log_posterior(Xt), ref.predict_joint_log_proba(Xt), rtol=1e-10, atol=1e-8)


def test_nearest_neighbour_matches_sklearn_and_brute_force():
    nbrs = pytest.importorskip("sklearn.neighbors")
    X, y = _data(11, n=150, d=5)
    Xt, _ = _data(12, n=80, d=5)
    ours = bl.NearestNeighbour().fit(X, y).predict(Xt)
    brute = np.array([y[int(np.argmin([np.sum((x - z) ** 2) for z in X]))] for x in Xt])
    assert np.array_equal(ours, brute)
    assert np.array_equal(ours, nbrs.KNeighborsClassifier(n_neighbors=1).fit(X, y).predict(Xt))


def test_stored_comparison_is_reproduced():
    """The committed comparison (every classifier on the committed table, both
    label sets) is what the code computes now, and the paper's tree reaches
    the 95 %-of-best mark on the held-out matrices."""
    from paper_1805_11938_gb300.train_selector import load_table

    recs = load_table(os.path.join(DATA, "corpus_table.jsonl"))
    with open(os.path.join(DATA, "selector_alternatives.json")) as f:
        stored = json.load(f)
    for key in ("ms", "ms_batch"):
        now = bl.compare(recs, key)
        for name, r in stored[key].items():
            assert abs(now[name]["mean_pct_of_best"] - r["mean_pct_of_best"]) < 1e-9, (key, name)
        assert now["DTC (the paper's)"]["mean_pct_of_best"] >= 95.0
