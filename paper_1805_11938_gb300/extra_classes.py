"""Plain SELL and standalone COO as extra selector classes: what seven classes
gain over the paper's five, measured on this GPU.

The paper's candidates are CSR, CSR5, ELL, SELL-C-sigma and HYB (Sec. III).
Its background also describes plain SELL (sigma = 1: slices of consecutive
rows, no sorting) and the standalone COO format; both are settings of the
library's kernels (SELL with sell_sigma = 1; HYB with every entry in its COO
part).  A corpus table profiled with seven classes (profile_corpus
--classes 7: all seven timed in the same run) answers two questions:

  * the oracle gain: how much faster the best of seven is than the best of
    the five (t_best5 / t_best7 per matrix), and how often an extra class is
    the fastest;
  * the selector gain: the paper's decision tree (and the 1-NN rule) trained
    on the seven-class labels against the same classifier trained on the
    five-class labels, both scored against the best of seven on the same
    held-out matrices (the split, features and measure of the shipped
    selector).

    python -m paper_1805_11938_gb300.extra_classes --table data/corpus_table7.jsonl \\
        --out data/selector_seven_classes.json
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

BASE = ("CSR", "CSR5", "ELL", "SELL", "HYB")


def best(ms: dict, names) -> tuple:
    """The fastest feasible class among `names` and its time."""
    feas = {k: ms[k] for k in names if ms.get(k) is not None}
    k = min(feas, key=lambda c: feas[c])
    return k, feas[k]


def pct_vs(ms: dict, names, chosen: str) -> float:
    """perf(chosen) / perf(best of `names`) = t_best / t_chosen; 0 if chosen is infeasible."""
    t = ms.get(chosen)
    return 0.0 if t is None else best(ms, names)[1] / t


def evaluate(records: list, key: str = "ms") -> dict:
    from .baselines import DecisionTree, NearestNeighbour, features_matrix
    from .train_selector import split

    names = list(records[0]["classes"])
    assert names[:len(BASE)] == list(BASE), names
    extra = names[len(BASE):]
    n = len(records)
    # the oracle: the best of seven against the best of five, every matrix
    b5 = [best(r[key], BASE) for r in records]
    b7 = [best(r[key], names) for r in records]
    gain = np.array([t5 / t7 for (_, t5), (_, t7) in zip(b5, b7)])
    counts = {c: sum(1 for k, _ in b7 if k == c) for c in names}
    out = {"matrices": n, "classes": names, "best_counts": counts,
           "extra_best_fraction": float(np.mean([k in extra for k, _ in b7])),
           "oracle_speedup_of_best7_over_best5": {"mean": float(gain.mean()), "max": float(gain.max()),
                                                   "geomean": float(np.exp(np.log(gain).mean()))},
           "best5_pct_of_best7_mean": 100 * float(np.mean(1.0 / gain))}
    # the classifiers, trained on the same training matrices
    tr, te = split(n, n_train=int(round(0.8 * n)))
    Xtr, Xte = features_matrix(records, tr), features_matrix(records, te)
    lo, hi = Xtr.min(axis=0), Xtr.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)

    def scaled(Z):
        return np.clip((Z - lo) / span, 0.0, 1.0)

    y5 = np.array([BASE.index(b5[i][0]) for i in tr])
    y7 = np.array([names.index(b7[i][0]) for i in tr])
    for label, classes, y in (("five_classes", BASE, y5), ("seven_classes", names, y7)):
        res = {}
        for mname, mdl, Xa, Xb in (("DTC (the paper's)", DecisionTree(n_classes=len(classes)), Xtr, Xte),
                                   ("KNC (k=1)", NearestNeighbour(), scaled(Xtr), scaled(Xte))):
            pred = mdl.fit(Xa, y).predict(Xb)
            r = np.array([pct_vs(records[i][key], names, classes[int(p)]) for i, p in zip(te, pred)])
            res[mname] = {"mean_pct_of_best7": 100 * float(r.mean()), "worst_pct_of_best7": 100 * float(r.min())}
        out[label] = res
    # what the shipped five classes can reach at best on the held-out matrices
    out["held_out_best5_pct_of_best7"] = 100 * float(np.mean([1.0 / gain[i] for i in te]))
    return out


def main():
    from .train_selector import load_table

    ap = argparse.ArgumentParser()
    ap.add_argument("--table", required=True)
    ap.add_argument("--out")
    args = ap.parse_args()
    recs = load_table(args.table)
    res = {key: evaluate(recs, key) for key in ("ms", "ms_batch")}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
