"""The paper's own selector and its alternatives, on the CPU, on the same features.

Sec. V-B builds the predictor as a decision tree (scikit-learn's
DecisionTreeClassifier: Gini impurity, grown until the leaves are pure);
Sec. V-D compares it with the other classifiers of Fig. 11: Gaussian naive
Bayes, the 1-nearest-neighbour rule, logistic regression, random forests and
a soft-voting / majority-rule ensemble (the multilayer perceptron of that
list is the library's own network).  They are written here from their
definitions (numpy; scipy's L-BFGS minimiser for logistic regression) and
trained and scored exactly like the library's network:
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


def best_split(X: np.ndarray, y: np.ndarray, n_classes: int = N_CLASSES, features=None):
    """The split (feature j, threshold t: left = x_j <= t) that minimises the
    sample-weighted Gini impurity of the two children, by exhaustive search
    over every feature (or the given ones, in the given order) and every
    boundary between distinct sorted values; the threshold is the midpoint of
    the two values.  Ties go to the earlier feature, then the lower threshold.
    None if no split separates."""
    n, d = X.shape
    best = None
    onehot = np.eye(n_classes, dtype=np.float64)[y]
    for j in (range(d) if features is None else features):
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
    (scikit-learn's defaults), optionally bounded by max_depth.  With
    max_features (random forests) each node draws the features to search in
    a random order from `rng` and stops once it has searched max_features of
    them and found a split (scikit-learn's rule: it searches on past
    max_features while no split has been found)."""

    def __init__(self, max_depth: int | None = None, n_classes: int = N_CLASSES, max_features: int | None = None,
                 rng=None):
        self.max_depth = max_depth
        self.n_classes = n_classes
        self.max_features = max_features
        self.rng = rng
        self.nodes = []  # (feature, threshold, left, right, label); feature -1 for a leaf
        self.leaf_counts = {}  # leaf node -> class counts of its training samples

    def fit(self, X: np.ndarray, y: np.ndarray) -> "DecisionTree":
        X = np.asarray(X, dtype=np.float64)
        y = np.asarray(y, dtype=np.int64)
        self.nodes = []
        self.leaf_counts = {}
        self._grow(X, y, 0)
        return self

    def _split(self, X, y):
        d = X.shape[1]
        if self.max_features is None or self.max_features >= d:
            return best_split(X, y, self.n_classes)
        order = self.rng.permutation(d)
        best = None
        for q in range(d):
            sp = best_split(X, y, self.n_classes, features=[int(order[q])])
            if sp is not None and (best is None or sp[2] < best[2] - 1e-15):
                best = sp
            if q + 1 >= self.max_features and best is not None:
                break
        return best

    def _grow(self, X, y, depth) -> int:
        counts = np.bincount(y, minlength=self.n_classes)
        label = int(np.argmax(counts))  # majority, ties to the lower class id
        k = len(self.nodes)
        self.nodes.append((-1, 0.0, -1, -1, label))
        self.leaf_counts[k] = counts
        if counts.max() == len(y) or (self.max_depth is not None and depth >= self.max_depth):
            return k
        sp = self._split(X, y)
        if sp is None or sp[2] >= _gini(counts.astype(np.float64)) - 1e-15:
            return k
        j, t, _ = sp
        del self.leaf_counts[k]
        m = X[:, j] <= t
        left = self._grow(X[m], y[m], depth + 1)
        right = self._grow(X[~m], y[~m], depth + 1)
        self.nodes[k] = (j, t, left, right, label)
        return k

    def _leaf(self, x) -> int:
        k = 0
        while self.nodes[k][0] >= 0:
            j, t, left, right, _ = self.nodes[k]
            k = left if x[j] <= t else right
        return k

    def predict(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        return np.array([self.nodes[self._leaf(x)][4] for x in X], dtype=np.int64)

    def predict_proba(self, X: np.ndarray) -> np.ndarray:
        """Class fractions of the training samples in each sample's leaf."""
        X = np.asarray(X, dtype=np.float64)
        out = np.empty((len(X), self.n_classes))
        for i, x in enumerate(X):
            c = self.leaf_counts[self._leaf(x)].astype(np.float64)
            out[i] = c / c.sum()
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

    def predict_proba(self, X) -> np.ndarray:
        """Posterior probabilities over all n_classes (0 for a class absent from training)."""
        lp = self.log_posterior(X)
        p = np.exp(lp - lp.max(axis=1, keepdims=True))
        out = np.zeros((len(p), self.n_classes))
        out[:, self.classes] = p / p.sum(axis=1, keepdims=True)
        return out


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

    def predict_proba(self, X) -> np.ndarray:
        """The neighbour's label as a one-hot distribution."""
        return np.eye(N_CLASSES)[self.predict(X)]


# ------------------------------------------------------ logistic regression

class LogisticRegression:
    """Multinomial logistic regression: class scores z = X W + b, softmax
    probabilities, minimising C * (summed cross-entropy) + ||W||^2 / 2 (the
    intercept b unpenalised), scikit-learn's objective with its default
    C = 1.  The exact objective and gradient go to scipy's L-BFGS-B."""

    def __init__(self, C: float = 1.0, n_classes: int = N_CLASSES, tol: float = 1e-10, max_iter: int = 20000):
        self.C, self.n_classes, self.tol, self.max_iter = C, n_classes, tol, max_iter

    def _unpack(self, w, d):
        k = self.n_classes
        return w[:d * k].reshape(d, k), w[d * k:]

    def objective(self, w, X, y):
        """(value, gradient) of the penalised loss at the flat parameters w."""
        n, d = X.shape
        W, b = self._unpack(w, d)
        z = X @ W + b
        z = z - z.max(axis=1, keepdims=True)
        lse = np.log(np.exp(z).sum(axis=1))
        loss = float(lse.sum() - z[np.arange(n), y].sum())
        p = np.exp(z - lse[:, None])
        p[np.arange(n), y] -= 1.0
        gW = self.C * (X.T @ p) + W
        gb = self.C * p.sum(axis=0)
        return self.C * loss + 0.5 * float((W * W).sum()), np.concatenate([gW.ravel(), gb])

    def fit(self, X, y) -> "LogisticRegression":
        from scipy.optimize import minimize

        X = np.asarray(X, dtype=np.float64)
        y = np.asarray(y, dtype=np.int64)
        d = X.shape[1]
        w0 = np.zeros(d * self.n_classes + self.n_classes)
        r = minimize(self.objective, w0, args=(X, y), jac=True, method="L-BFGS-B",
                     options={"maxiter": self.max_iter, "gtol": self.tol, "ftol": 0.0})
        self.W, self.b = self._unpack(r.x, d)
        self.converged = bool(r.success)
        return self

    def predict_proba(self, X) -> np.ndarray:
        z = np.asarray(X, dtype=np.float64) @ self.W + self.b
        z = z - z.max(axis=1, keepdims=True)
        e = np.exp(z)
        return e / e.sum(axis=1, keepdims=True)

    def predict(self, X) -> np.ndarray:
        return np.argmax(self.predict_proba(X), axis=1)


# ----------------------------------------------------------- random forests

class RandomForest:
    """Random forests: n_trees CART trees, each grown fully on a bootstrap
    sample (n draws with replacement) with max_features = floor(sqrt(d))
    features searched per node; the forest predicts the class of the largest
    mean leaf-class fraction over the trees (scikit-learn's rule, ties to the
    lower class id).  Seeded: the same seed grows the same forest."""

    def __init__(self, n_trees: int = 100, max_features: int | None = None, bootstrap: bool = True, seed: int = 0,
                 n_classes: int = N_CLASSES):
        self.n_trees, self.max_features, self.bootstrap = n_trees, max_features, bootstrap
        self.seed, self.n_classes = seed, n_classes

    def fit(self, X, y) -> "RandomForest":
        X = np.asarray(X, dtype=np.float64)
        y = np.asarray(y, dtype=np.int64)
        n, d = X.shape
        mf = self.max_features if self.max_features is not None else max(1, int(np.sqrt(d)))
        rng = np.random.default_rng(self.seed)
        self.trees = []
        for _ in range(self.n_trees):
            rows = rng.integers(0, n, size=n) if self.bootstrap else np.arange(n)
            t = DecisionTree(n_classes=self.n_classes, max_features=mf, rng=rng).fit(X[rows], y[rows])
            self.trees.append(t)
        return self

    def predict_proba(self, X) -> np.ndarray:
        return np.mean([t.predict_proba(X) for t in self.trees], axis=0)

    def predict(self, X) -> np.ndarray:
        return np.argmax(self.predict_proba(X), axis=1)


# ------------------------------------------------------------------- voting

class Voting:
    """An ensemble of fitted classifiers.  "soft": the class of the largest
    mean predicted probability; "hard" (majority rule): the class most of
    them predict, ties to the lower class id."""

    def __init__(self, members: list, voting: str = "soft", n_classes: int = N_CLASSES):
        if voting not in ("soft", "hard"):
            raise ValueError("voting is 'soft' or 'hard'")
        self.members, self.voting, self.n_classes = members, voting, n_classes

    def predict(self, Xs) -> np.ndarray:
        """Xs: one input matrix per member (members may see differently scaled features)."""
        if self.voting == "soft":
            return np.argmax(np.mean([m.predict_proba(X) for m, X in zip(self.members, Xs)], axis=0), axis=1)
        votes = np.stack([m.predict(X) for m, X in zip(self.members, Xs)], axis=1)
        counts = np.stack([(votes == c).sum(axis=1) for c in range(self.n_classes)], axis=1)
        return np.argmax(counts, axis=1)


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

    dtc = DecisionTree().fit(Xtr, ytr)
    gnb = GaussianNB().fit(Xtr, ytr)
    knc = NearestNeighbour().fit(scaled(Xtr), ytr)
    lr = LogisticRegression().fit(scaled(Xtr), ytr)
    rfc = RandomForest(seed=0).fit(Xtr, ytr)
    members = [dtc, gnb, knc, lr, rfc]
    Xs = [Xte, Xte, scaled(Xte), scaled(Xte), Xte]  # each member's own inputs
    preds = {name: m.predict(X) for name, m, X in zip(("DTC (the paper's)", "GNB", "KNC (k=1)", "LR", "RFC"), members, Xs)}
    # the ensemble of the five: soft voting averages the tree's leaf
    # fractions, GNB's posterior, the neighbour's one-hot vote, LR's and the
    # forest's probabilities; majority rule counts their predictions
    preds["VC (soft)"] = Voting(members, "soft").predict(Xs)
    preds["VC (majority)"] = Voting(members, "hard").predict(Xs)
    out = {}
    models = {"DTC (the paper's)": dtc}
    for name, pred in preds.items():
        mdl = models.get(name)
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
