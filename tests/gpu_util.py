"""Helpers shared by the GPU parity tests (no test functions here)."""
import numpy as np

import oracle
import synth


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def within_bound(a, x, y):
    """|y_i - y_ref,i| <= 4 * nnz_i * 2^-53 * sum_j |a_ij x_j| for every row (the FP64 tolerance)."""
    ref = oracle.csr_spmv(a, x)
    b = oracle.fp_bound(a, x)
    err = np.abs(np.asarray(y) - ref)
    ok = err <= b
    if not ok.all():
        i = int(np.argmax(~ok))
        return False, f"row {i}: y={y[i]!r} ref={ref[i]!r} err={err[i]:.3e} bound={b[i]:.3e}"
    return True, ""


def row_subset(a, rows):
    """CSR of the given rows only (for sampled checks at full size)."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = (a.ptr[rows + 1] - a.ptr[rows]).astype(np.int64)
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    idx = np.concatenate([a.idx[a.ptr[r]:a.ptr[r + 1]] for r in rows]) if len(rows) else np.zeros(0, np.int32)
    val = np.concatenate([a.val[a.ptr[r]:a.ptr[r + 1]] for r in rows]) if len(rows) else np.zeros(0)
    return synth.CSR(len(rows), a.n, ptr, idx.astype(np.int32), val, a.name + "_rows")


def matrices_small():
    """Small and ragged cases that still span several units, tiles and slices."""
    out = [
        synth.config1(),
        synth.powerlaw(20_000, 101, xmax=3000, lmax=3000),           # long rows, split chunks
        synth.powerlaw(3_001, 102, xmax=60, lmax=60),                 # ragged tail
        synth.banded(5_000, 9, 103),
        synth.stencil(synth.STENCIL_27PT_3D, 13, 11, 7, 104),
        synth.blockdiag(4_099, 33, 105),
        synth.uniform_random(2_500, 17, 106),
        synth.tiny_random(7, 5, 0.5, 107),
        synth.tiny_random(1, 1, 1.0, 108),
    ]
    # empty rows interleaved with long ones
    lens = np.array([0, 0, 5000, 0, 3, 0, 0, 70, 1, 0] * 300, dtype=np.int32)
    out.append(synth.from_lengths_random_cols(lens, 6000, 109, "empty_mix"))
    # one dense row much longer than a CSR chunk, rest empty
    lens = np.zeros(64, np.int32)
    lens[31] = 60_000
    out.append(synth.from_lengths_random_cols(lens, 60_000, 110, "one_long_row"))
    # CSR tiles hold 352 nonzeros: rows starting on tile boundaries, spanning two and three
    # tiles, overflowing the next tile by exactly one tile and by one more, empty rows around
    lens = np.array([0, 352, 352, 351, 1, 353, 704, 1, 0, 351, 353, 351, 354, 0, 0], dtype=np.int32)
    out.append(synth.from_lengths_random_cols(lens, 900, 111, "tile_edges"))
    # nonzeros an exact multiple of 352, trailing empty rows
    lens = np.array([0, 0, 352, 0, 352, 0, 0], dtype=np.int32)
    out.append(synth.from_lengths_random_cols(lens, 500, 112, "tile_exact"))
    return out
