"""The seeded input generators against closed forms: the structured families'
patterns are fixed by their definitions (a stencil's in-grid neighbours, a
band, dense diagonal blocks), so their sizes and columns are checked exactly;
the workload configurations have the sizes the measurements quote."""
import numpy as np
import pytest

import synth


def _brute_stencil(kind, nx, ny, nz):
    offs = {synth.STENCIL_5PT_2D: [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)],
            synth.STENCIL_9PT_2D: [(a, b, 0) for a in (-1, 0, 1) for b in (-1, 0, 1)],
            synth.STENCIL_7PT_3D: [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)],
            synth.STENCIL_27PT_3D: [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]}[kind]
    rows = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                cols = sorted((z + c) * nx * ny + (y + b) * nx + (x + a) for a, b, c in offs
                              if 0 <= x + a < nx and 0 <= y + b < ny and 0 <= z + c < nz)
                rows.append(cols)
    return rows


@pytest.mark.parametrize("kind,nx,ny,nz", [(synth.STENCIL_5PT_2D, 7, 5, 1), (synth.STENCIL_9PT_2D, 6, 4, 1),
                                           (synth.STENCIL_7PT_3D, 4, 3, 5), (synth.STENCIL_27PT_3D, 4, 5, 3)])
def test_stencil_pattern_is_the_in_grid_neighbours(kind, nx, ny, nz):
    ptr, idx = synth.stencil_pattern(kind, nx, ny, nz)
    rows = _brute_stencil(kind, nx, ny, nz)
    assert [sorted(idx[ptr[i]:ptr[i + 1]].tolist()) for i in range(len(rows))] == rows


def test_stencil_counts_closed_forms():
    for n in (2, 5, 9):
        assert synth.stencil_pattern(synth.STENCIL_27PT_3D, n, n, n)[0][-1] == (3 * n - 2) ** 3
        assert synth.stencil_pattern(synth.STENCIL_7PT_3D, n, n, n)[0][-1] == n ** 3 + 6 * n * n * (n - 1)
    for nx, ny in ((3, 8), (64, 64)):
        assert synth.stencil_pattern(synth.STENCIL_5PT_2D, nx, ny)[0][-1] == 5 * nx * ny - 2 * nx - 2 * ny
        assert synth.stencil_pattern(synth.STENCIL_9PT_2D, nx, ny)[0][-1] == (3 * nx - 2) * (3 * ny - 2)
    assert (3 * 224 - 2) ** 3 == 300_763_000  # the 224^3 stencil workload's nnz


def test_config1_is_the_64x64_laplacian():
    a = synth.config1()
    assert (a.m, a.n, int(a.ptr[-1])) == (4096, 4096, 20_224)


def test_banded_and_blockdiag_closed_forms():
    for n, bw in ((50, 3), (1000, 64), (7, 10)):
        a = synth.banded(n, bw, 1)
        b = min(bw, n - 1)
        assert int(a.ptr[-1]) == n * (2 * b + 1) - b * (b + 1)
        for i in (0, n // 2, n - 1):
            assert a.idx[a.ptr[i]:a.ptr[i + 1]].tolist() == list(range(max(0, i - bw), min(n, i + bw + 1)))
    for n, bs in ((100, 8), (99, 8), (5, 64)):
        a = synth.blockdiag(n, bs, 2)
        assert int(a.ptr[-1]) == (n // bs) * bs * bs + (n % bs) ** 2
        i = n - 1
        start = (i // bs) * bs
        assert a.idx[a.ptr[i]:a.ptr[i + 1]].tolist() == list(range(start, min(n, start + bs)))


def test_generators_are_seeded():
    a1, a2 = synth.powerlaw(5000, 77), synth.powerlaw(5000, 77)
    assert np.array_equal(a1.ptr, a2.ptr) and np.array_equal(a1.idx, a2.idx) and np.array_equal(a1.val, a2.val)
    b = synth.powerlaw(5000, 78)
    assert not np.array_equal(a1.idx[:100], b.idx[:100])
    assert np.array_equal(synth.vector(100, 3), synth.vector(100, 3))
