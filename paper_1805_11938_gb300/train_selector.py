"""Train and evaluate the format selector on the GPU with the library's kernels.

Sec. V-B: the classifier learns (features -> best representation) from the
profiled training matrices; features are min-max scaled with the training
set's extremes, which are stored with the model (Sec. V-B "Feature
Scaling").  Sec. V-C evaluates on held-out matrices the performance of the
predicted format relative to the best one found by exhaustive search.

Here the network is the 16-64-64-5 MLP; scaling (spmv_mlp_scale), the
full-batch Adam training loop (spmv_mlp_train) and inference
(spmv_mlp_forward) all run in this library's CUDA kernels.  The split is 800
training / 200 held-out matrices by a seeded shuffle.

Steps and learning rate are chosen by five-fold cross-validation on the 800
training matrices (the paper trains with five-fold cross-validation); the
held-out 200 play no part in the choice.

Two models come from one profiling table: --key ms learns the fastest format
for one product of a matrix alone (spmv_select's model), --key ms_batch the
format with the best throughput when the GPU is kept busy, as in a batch
(the model that picks formats for spmv_batch).

    python -m paper_1805_11938_gb300.train_selector --table table.jsonl --out model.json [--key ms_batch]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FORMATS = ("CSR", "CSR5", "ELL", "SELL", "HYB")
LAYERS = ((16, 64), (64,), (64, 64), (64,), (64, 5), (5,))
LOG_FEATURES = (0, 1, 3, 4, 5, 6, 11, 12)


def load_table(path: str) -> list:
    recs = {}
    with open(path) as f:
        for line in f:
            r = json.loads(line)
            recs[r["index"]] = r
    return [recs[i] for i in sorted(recs)]


def split(n: int, n_train: int = 800, seed: int = 0):
    """Seeded shuffle of 0..n-1: the first n_train are training matrices, the rest held out."""
    import synth

    keys = np.array([synth.u01(seed, 0x5B117, i) for i in range(n)])
    order = np.argsort(keys, kind="stable")
    return np.sort(order[:n_train]), np.sort(order[n_train:])


def transform(f: np.ndarray) -> np.ndarray:
    """The feature transform the device applies before scaling (used here only to fit lo/hi)."""
    t = np.array(f, dtype=np.float64, copy=True)
    for j in LOG_FEATURES:
        t[..., j] = np.log2(1.0 + t[..., j])
    t[..., 2] = -np.log2(np.maximum(t[..., 2], 2.0 ** -60))
    return t


def init_params(seed: int) -> np.ndarray:
    """Glorot-uniform weights from the seeded generator, zero biases."""
    import synth

    u = synth.vector(sum(int(np.prod(s)) for s in LAYERS), seed)
    out, o = [], 0
    for s in LAYERS:
        k = int(np.prod(s))
        if len(s) == 2:
            out.append(u[o:o + k] * math.sqrt(6.0 / (s[0] + s[1])))
        else:
            out.append(np.zeros(k))
        o += k
    return np.concatenate(out).astype(np.float32)


def _dev(a, dtype=None):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a)).cuda() if dtype is None else torch.as_tensor(np.ascontiguousarray(a, dtype=dtype)).cuda()


LABEL_OF = {"ms": "label", "ms_batch": "label_batch"}


def fit(records: list, train_idx, steps: int = 3000, lr: float = 3e-3, seed: int = 1, key: str = "ms") -> dict:
    import torch

    from . import spmv_mlp_scale, spmv_mlp_train

    F = np.array([records[i]["features"] for i in train_idx], dtype=np.float32)
    labels = np.array([records[i][LABEL_OF[key]] for i in train_idx], dtype=np.int32)
    t = transform(F.astype(np.float64))
    lo, hi = t.min(axis=0).astype(np.float32), t.max(axis=0).astype(np.float32)
    X = spmv_mlp_scale(_dev(F), _dev(lo), _dev(hi))
    theta = _dev(init_params(seed))
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    hist = spmv_mlp_train(theta, m, v, X, _dev(labels), steps, 0, lr=lr).cpu().numpy()
    return {"params": theta.cpu().numpy(), "lo": lo, "hi": hi, "loss_first": float(hist[0]),
            "loss_last": float(hist[-1]), "steps": steps, "lr": lr, "seed": seed}


def predict(model: dict, records: list, idx) -> np.ndarray:
    from . import spmv_mlp_forward, spmv_mlp_scale

    F = np.array([records[i]["features"] for i in idx], dtype=np.float32)
    X = spmv_mlp_scale(_dev(F), _dev(model["lo"], np.float32), _dev(model["hi"], np.float32))
    _, pred = spmv_mlp_forward(_dev(model["params"], np.float32), X)
    return pred.cpu().numpy()


def pct_of_best(records: list, idx, choice, key: str = "ms") -> np.ndarray:
    """perf(chosen) / perf(best) = t_best / t_chosen per matrix (0 if the chosen format is infeasible)."""
    out = []
    for i, c in zip(idx, choice):
        ms = records[i][key]
        best = min(v for v in ms.values() if v is not None)
        t = ms[FORMATS[int(c)]]
        out.append(0.0 if t is None else best / t)
    return np.array(out)


def summary(records: list, idx, pred, key: str = "ms") -> dict:
    r = pct_of_best(records, idx, pred, key)
    out = {"mean_pct_of_best": 100 * float(r.mean()), "geomean_pct_of_best": 100 * float(np.exp(np.log(np.maximum(r, 1e-9)).mean())),
           "worst_pct_of_best": 100 * float(r.min()),
           "accuracy": float(np.mean([records[i][LABEL_OF[key]] == int(p) for i, p in zip(idx, pred)])), "n": len(idx)}
    fixed = {FORMATS[f]: 100 * float(pct_of_best(records, idx, [f] * len(idx), key).mean()) for f in range(5)}
    out["fixed_format_mean_pct_of_best"] = fixed
    out["best_fixed_format"] = max(fixed, key=fixed.get)
    out["gain_over_best_fixed_pct_points"] = out["mean_pct_of_best"] - fixed[out["best_fixed_format"]]
    out["gain_over_always_csr_pct_points"] = out["mean_pct_of_best"] - fixed["CSR"]
    return out


SETTINGS = tuple({"steps": st, "lr": lr} for st in (1500, 3000, 6000) for lr in (1e-3, 3e-3, 1e-2))


def cross_validate(records: list, train_idx, key: str = "ms", folds: int = 5, settings=SETTINGS, seed: int = 1):
    """Five-fold cross-validation on the training matrices only (Sec. V-B):
    for each setting, the mean over the folds of the held-in-fold % of best;
    returns (best setting, table).  Ties go to the earlier setting."""
    train_idx = np.asarray(train_idx)
    parts = np.array_split(train_idx, folds)
    table = []
    for st in settings:
        scores = []
        for f in range(folds):
            val = parts[f]
            fit_idx = np.concatenate([parts[g] for g in range(folds) if g != f])
            model = fit(records, fit_idx, st["steps"], st["lr"], seed, key)
            scores.append(float(pct_of_best(records, val, predict(model, records, val), key).mean()))
        table.append({**st, "cv_mean_pct_of_best": 100 * float(np.mean(scores))})
    best = max(range(len(table)), key=lambda i: (table[i]["cv_mean_pct_of_best"], -i))
    return settings[best], table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--table", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--key", default="ms", choices=sorted(LABEL_OF))
    ap.add_argument("--no-cv", action="store_true", help="train with --steps/--lr instead of choosing them by CV")
    args = ap.parse_args()
    recs = load_table(args.table)
    assert [r["index"] for r in recs] == list(range(len(recs))), "table must hold matrices 0..n-1"
    tr, te = split(len(recs), n_train=int(round(0.8 * len(recs))))
    cv = None
    if not args.no_cv:
        chosen, table = cross_validate(recs, tr, args.key, seed=args.seed)
        args.steps, args.lr = chosen["steps"], chosen["lr"]
        cv = {"folds": 5, "chosen": chosen, "table": table}
    model = fit(recs, tr, args.steps, args.lr, args.seed, args.key)
    ev_train = summary(recs, tr, predict(model, recs, tr), args.key)
    ev_test = summary(recs, te, predict(model, recs, te), args.key)
    out = {"params": model["params"].tolist(), "lo": model["lo"].tolist(), "hi": model["hi"].tolist(),
           "features": "spmv_features v3 (16 features; row-length statistics exact, histogram and index spread from 8192 rows sampled above 8192)",
           "timing": args.key, "cross_validation": cv,
           "training": {k: model[k] for k in ("steps", "lr", "seed", "loss_first", "loss_last")},
           "n_train": len(tr), "n_test": len(te), "train": ev_train, "held_out": ev_test}
    with open(args.out, "w") as f:
        json.dump(out, f)
    print(json.dumps({"train": ev_train, "held_out": ev_test, "training": out["training"]}, indent=1))


if __name__ == "__main__":
    main()
