"""The autotuner's repetition rule on the host: the paper's training-data rule
(repeat until the 95 % confidence interval of the mean is narrower than 5 % of
the mean), with the Student-t quantiles it uses pinned to scipy's."""
import math

import numpy as np
import pytest

from paper_1805_11938_gb300 import autotune

scipy_stats = pytest.importorskip("scipy.stats")


def test_t_quantiles_match_scipy():
    for n in range(2, 11):  # the table: n samples, n - 1 degrees of freedom
        assert autotune._t95(n) == pytest.approx(scipy_stats.t.ppf(0.975, n - 1), abs=0.01)
    for n in (11, 15, 20, 40, 100, 200):  # the approximation beyond the table
        assert autotune._t95(n) == pytest.approx(scipy_stats.t.ppf(0.975, n - 1), rel=0.01)


class _FakeTimer(autotune.Timer):
    """Timer whose batches come from a list instead of CUDA events."""

    def __init__(self, times):
        self.times = list(times)
        self.calls = []

    def batch(self, fn, n):
        self.calls.append(n)
        out, self.times = self.times[:n], self.times[n:]
        return out


def test_steady_times_stop_at_the_minimum():
    t = _FakeTimer([1.0] * 50)
    r = t.measure(lambda: None, warmup=0, n_min=10)
    assert r["n"] == 10 and r["ms"] == 1.0 and r["ci_halfwidth_ms"] == 0.0 and t.calls == [10]


def test_noisy_times_repeat_until_the_interval_is_narrow():
    rng = np.random.default_rng(3)
    times = list(1.0 + 0.1 * rng.standard_normal(400))
    t = _FakeTimer(times)
    r = t.measure(lambda: None, warmup=0, n_min=10, n_max=400)
    xs = times[:r["n"]]
    half = autotune._t95(len(xs)) * np.std(xs, ddof=1) / math.sqrt(len(xs))
    assert r["ci_halfwidth_ms"] == pytest.approx(half)
    assert 2 * half <= 0.05 * np.mean(xs)  # the rule holds where it stopped
    n_prev = r["n"] - t.calls[-1]          # and did not hold one batch earlier
    prev = times[:n_prev]
    assert 2 * autotune._t95(n_prev) * np.std(prev, ddof=1) / math.sqrt(n_prev) > 0.05 * np.mean(prev)


def test_very_noisy_times_stop_at_the_maximum():
    t = _FakeTimer([1.0, 3.0] * 200)
    r = t.measure(lambda: None, warmup=0, n_min=10, n_max=60)
    assert r["n"] >= 60 and r["n"] - t.calls[-1] < 60
