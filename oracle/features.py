"""CPU ORACLE (test infrastructure only): the selector's 16 matrix features.

Sec. V-B "Features" / Table IV: static features of the matrix alone, no
profiling -- n_rows, n_cols, nnz_frac, nnz_min, nnz_max, nnz_avg, nnz_std and
"variation".  Eight more are added for the GPU formats.  Definitions (the paper
gives names only; the readings are ours):

len_i = ptr[i+1] - ptr[i] over all rows i < M; nnz = ptr[M] = sum of len_i.
Row sample R (for features 10, 11, 12 and 15 only): all rows if M <= 8192,
else rows floor(k*M/8192), k < 8192; L = sum over R of len_i.

 0 n_rows      M
 1 n_cols      N
 2 nnz_frac    nnz / (M*N)
 3 nnz_min     min over all rows of len_i
 4 nnz_max     max over all rows of len_i
 5 nnz_avg     nnz / M
 6 nnz_std     population std of len over all rows: sqrt(M*sum len^2 - nnz^2) / M
 7 variation   nnz_std / nnz_avg, 0 if nnz = 0  (coefficient of variation)
 8 log2_nnz    log2(max(nnz, 1))
 9 ell_fill    nnz_avg / nnz_max, 0 if nnz_max = 0
10 hyb_tail    sum over R of max(0, len_i - K) / L, 0 if L = 0, where K is the
               HYB rule on R with lengths capped at 512: the largest
               k in [1, 512] with #{len_i >= k} >= ceil(|R|/3), else 0
11 diag_spread mean |col - i| over the first min(len_i, 16) entries of each
               sampled row (0 if none)
12 bandwidth   max |col - i| over the same entries
13 empty_frac  #{len_i = 0} / M
14 long_frac   #{len_i >= 32} / M
15 sell32_fill fill of SELL-32 with rows sorted over all of R, lengths capped
               at 512: sum min(len_i, 512) / (32 * sum_{k=1..512} ceil(c_k/32)),
               c_k = #{len_i >= k} over R; 1 if the denominator is 0.  (Slice s
               of the descending order has width >= k exactly when 32*s < c_k.)
"""
from __future__ import annotations

import math

import numpy as np

FEATURE_NAMES = ("n_rows", "n_cols", "nnz_frac", "nnz_min", "nnz_max", "nnz_avg", "nnz_std", "variation",
                 "log2_nnz", "ell_fill", "hyb_tail", "diag_spread", "bandwidth", "empty_frac", "long_frac",
                 "sell32_fill")
SAMPLE_ROWS = 8192
LEN_CAP = 512
SPREAD_ENTRIES = 16
LONG_ROW = 32


def sample_rows(m: int) -> list[int]:
    s = min(m, SAMPLE_ROWS)
    return [(k * m) // s for k in range(s)]


def hyb_k_of_lengths(lengths, cap: int | None = None) -> int:
    """Largest k (<= cap if given) such that at least ceil(|lengths|/3) lengths are >= k; 0 if none."""
    n = len(lengths)
    if n == 0:
        return 0
    need = -(-n // 3)
    top = max(lengths) if cap is None else min(max(lengths), cap)
    hist = [0] * (top + 1)
    for l in lengths:
        hist[min(l, top)] += 1
    at_least = 0
    for k in range(top, 0, -1):
        at_least += hist[k]
        if at_least >= need:
            return k
    return 0


def features(a) -> np.ndarray:
    """The 16 features of CSR matrix `a` as float64 (the device rounds them to float32)."""
    m, n = a.m, a.n
    ptr = [int(v) for v in a.ptr]
    nnz = ptr[m]
    # whole-matrix row-length statistics, exact integers (the sum of squares is
    # at most nnz * max len < 2^62, so int64 holds it)
    all_lens = np.diff(np.asarray(a.ptr, dtype=np.int64))
    sq = int(np.sum(all_lens * all_lens))
    std = math.sqrt(m * sq - nnz * nnz) / m  # Python integers, one rounding inside sqrt's argument
    mean = nnz / m
    mx = int(all_lens.max())
    # the sampled rows
    rows = sample_rows(m)
    lens = [ptr[i + 1] - ptr[i] for i in rows]
    L = sum(lens)
    K = hyb_k_of_lengths(lens, LEN_CAP)
    tail = sum(max(0, l - K) for l in lens)
    spread_sum, spread_cnt, band = 0, 0, 0
    idx = a.idx
    for i in rows:
        for k in range(ptr[i], ptr[i] + min(ptr[i + 1] - ptr[i], SPREAD_ENTRIES)):
            d = abs(int(idx[k]) - i)
            spread_sum += d
            spread_cnt += 1
            band = max(band, d)
    at_least = [0] * (LEN_CAP + 2)  # at_least[k] = #{len_i >= k}, lengths capped at LEN_CAP
    for l in lens:
        at_least[min(l, LEN_CAP)] += 1
    for k in range(LEN_CAP - 1, -1, -1):
        at_least[k] += at_least[k + 1]
    slice_widths = sum(-(-at_least[k] // 32) for k in range(1, LEN_CAP + 1))
    capped = sum(min(l, LEN_CAP) for l in lens)
    f = [
        float(m),
        float(n),
        nnz / (m * n),
        float(all_lens.min()),
        float(mx),
        mean,
        std,
        std / mean if nnz > 0 else 0.0,
        math.log2(max(nnz, 1)),
        mean / mx if mx > 0 else 0.0,
        tail / L if L > 0 else 0.0,
        spread_sum / spread_cnt if spread_cnt > 0 else 0.0,
        float(band),
        int(np.count_nonzero(all_lens == 0)) / m,
        int(np.count_nonzero(all_lens >= LONG_ROW)) / m,
        capped / (32 * slice_widths) if slice_widths > 0 else 1.0,
    ]
    return np.array(f, dtype=np.float64)
