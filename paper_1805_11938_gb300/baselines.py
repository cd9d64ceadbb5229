"""The paper's own selector and its alternatives, on the CPU, on the same features.

Sec. V-B builds the predictor as a decision tree (scikit-learn's
DecisionTreeClassifier: Gini impurity, grown until the leaves are pure);
Sec. V-D compares it with other classifiers, among them Gaussian naive Bayes
and the 1-nearest-neighbour rule.  They are written here from their
definitions (numpy) and trained and scored exactly like the library's network:
the same 16 features after the same transform, the same 800/200 split, the
same measure (performance of the predicted format relative to the
exhaustively best one, Sec. V-C).  The network remains the selector the
library ships; these show what it gains over the paper's model.

    python -m paper_1805_11938_gb300.baselines --table data/corpus_table.jsonl --out data/selector_alternatives.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_CLASSES = 5


# ------------------------------------------------------------ decision tree

def _gini(counts: np.ndarray) -> np.ndarray:
    """Gini impurity 1 - sum p_c^2 of class-count rows (0 for empty rows)."""
    n = counts.sum(axis=-1, keepdims=True)
    p = np.divide(counts, n, out=np.zeros_like(counts, dtype=np.float64), where=n > 0)
    return 1.0 - (p * p).sum(axis=-1)


def best_split(X: np.ndarray, y: np.ndarray, n_classes: int = N_CLASSES):
    """The split (feature j, threshold t: left = x_j <= t) that minimises the
    sample-weighted Gini impurity of the two children, by exhaustive search
    over every feature and every boundary between distinct sorted values;
    the threshold is the midpoint of the two values.  Ties go to the lower
    feature index, then the lower threshold.  None if no split separates."""
    n, d = X.shape
    best = None
    onehot = np.eye(n_classes, dtype=np.float64)[y]
    for j in range(d):
        order = np.argsort(X[:, j], kind="stable")
        xs = X[order, j]
        left = np.cumsum(onehot[order], axis=0)[:-1]  # counts of the first i+1 samples
        right = left[-1] + onehot[order[-1]] - left if n > 1 else left
        valid = xs[1:] > xs[:-1]  # a boundary between distinct values
        if not valid.any():
            continue
        nl = np.arange(1, n, dtype=np.float64)
        imp = (nl * _gini(left) + (n - nl) * _gini(right)) / n
        imp = np.where(valid, imp, np.inf)
        i = int(np.argmin(imp))  # the first minimum: the lowest threshold
        if best is None or imp[i] < best[0] - 1e-15:
            best = (float(imp[i]), j, 0.5 * (xs[i] + xs[i + 1]))
    return None if best is None else (best[1], best[2], best[0])


class DecisionTree:
    """CART classifier: grows until every leaf is pure or cannot be split
    (scikit-learn's defaults), optionally bounded by max_depth."""

    def __init__(self, max_depth: int | None = None, n_classes: int = N_CLASSES):
        self.max_depth = max_depth
        self.n_classes = n_classes
        self.nodes = []  # (feature, threshold, left, right, label); feature -1 for a leaf

    def fit(self, X: np.ndarray, y: np.ndarray) -> "DecisionTree":
        X = np.asarray(X, dtype=np.float64)
        y = np.asarray(y, dtype=np.int64)
        self.nodes = []
        self._grow(X, y, 0)
        return self

    def _grow(self, X, y, depth) -> int:
        counts = np.bincount(y, minlength=self.n_classes)
        label = int(np.argmax(counts))  # majority, ties to the lower class id
        k = len(self.nodes)
        self.nodes.append((-1, 0.0, -1, -1, label))
        if counts.max() == len(y) or (self.max_depth is not None and depth >= self.max_depth):
            return k
        sp = best_split(X, y, self.n_classes)
        if sp is None or sp[2] >= _gini(counts.astype(np.float64)) - 1e-15:
            return k
        j, t, _ = sp
        m = X[:, j] <= t
        left = self._grow(X[m], y[m], depth + 1)
        right = self._grow(X[~m], y[~m], depth + 1)
        self.nodes[k] = (j, t, left, right, label)
        return k

    def predict(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        out = np.empty(len(X), dtype=np.int64)
        for i, x in enumerate(X):
            k = 0
            while self.nodes[k][0] >= 0:
                j, t, left, right, _ = self.nodes[k]
                k = left if x[j] <= t else right
            out[i] = self.nodes[k][4]
        return out

    def depth(self) -> int:
        def d(k):
            j, _, l, r, _ = self.nodes[k]
            return 0 if j < 0 else 1 + max(d(l), d(r))

        return d(0)


# ------------------------------------------------------- Gaussian naive Bayes

class GaussianNB:
    """Class priors and per-class, per-feature normal densities; the variances
    get epsilon = 1e-9 x the largest feature variance added (scikit-learn's
    var_smoothing).  Predicts the class of highest log posterior."""

    def __init__(self, var_smoothing: float = 1e-9, n_classes: int = N_CLASSES):
        self.var_smoothing = var_smoothing
        self.n_classes = n_classes

    def fit(self, X, y) -> "GaussianNB":
        X = np.asarray(X, dtype=np.float64)
        y = np.asarray(y, dtype=np.int64)
        eps = self.var_smoothing * X.var(axis=0).max()
        self.classes = np.unique(y)
        self.mu = np.array([X[y == c].mean(axis=0) for c in self.classes])
        self.var = np.array([X[y == c].var(axis=0) for c in self.classes]) + eps
        self.logprior = np.log(np.array([(y == c).mean() for c in self.classes]))
        return self

    def log_posterior(self, X) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        ll = -0.5 * (np.log(2 * np.pi * self.var)[None, :, :] + (X[:, None, :] - self.mu[None]) ** 2 / self.var[None])
        return self.logprior[None, :] + ll.sum(axis=2)

    def predict(self, X) -> np.ndarray:
        return self.classes[np.argmax(self.log_posterior(X), axis=1)]


# -------------------------------------------------------- nearest neighbour

class NearestNeighbour:
    """The 1-nearest-neighbour rule (Euclidean distance; ties to the earlier
    training sample)."""

    def fit(self, X, y) -> "NearestNeighbour":
        self.X = np.asarray(X, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.int64)
        return self

    def predict(self, X) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        d2 = ((X[:, None, :] - self.X[None, :, :]) ** 2).sum(axis=2)
        return self.y[np.argmin(d2, axis=1)]


# --------------------------------------------------------------- evaluation

def features_matrix(records, idx) -> np.ndarray:
    from .train_selector import transform

    return transform(np.array([records[i]["features"] for i in idx], dtype=np.float32).astype(np.float64))


def compare(records, key: str = "ms") -> dict:
    """Held-out % of best for each classifier, trained on the same 800 matrices."""
    from .train_selector import LABEL_OF, pct_of_best, split

    tr, te = split(len(records), n_train=int(round(0.8 * len(records))))
    Xtr, Xte = features_matrix(records, tr), features_matrix(records, te)
    ytr = np.array([records[i][LABEL_OF[key]] for i in tr])
    lo, hi = Xtr.min(axis=0), Xtr.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)

    def scaled(Z):
        return np.clip((Z - lo) / span, 0.0, 1.0)

    models = {"DTC (the paper's)": DecisionTree().fit(Xtr, ytr), "GNB": GaussianNB().fit(Xtr, ytr),
              "KNC (k=1)": NearestNeighbour().fit(scaled(Xtr), ytr)}
    out = {}
    for name, mdl in models.items():
        pred = mdl.predict(scaled(Xte) if name.startswith("KNC") else Xte)
        r = pct_of_best(records, te, pred, key)
        out[name] = {"mean_pct_of_best": 100 * float(r.mean()), "worst_pct_of_best": 100 * float(r.min()),
                     "accuracy": float(np.mean(pred == np.array([records[i][LABEL_OF[key]] for i in te])))}
        if isinstance(mdl, DecisionTree):
            out[name]["depth"] = mdl.depth()
            out[name]["nodes"] = len(mdl.nodes)
    return out


def main():
    from .train_selector import load_table

    ap = argparse.ArgumentParser()
    ap.add_argument("--table", required=True)
    ap.add_argument("--out", help="write both label sets' comparison here (JSON)")
    args = ap.parse_args()
    recs = load_table(args.table)
    res = {key: compare(recs, key) for key in ("ms", "ms_batch")}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
