"""The per-rank product of the row-partitioned split on the GPU: every rank's
block converted and multiplied by the library (here all ranks in one process
on one device, no collective), the blocks' y concatenated in rank order equal
to the oracle's product of the whole matrix -- bit for bit on integer inputs,
within the FP64 bound otherwise."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import bits, within_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    return m


@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("fmt", [0, 1, 3, 4])
def test_row_blocks_reassemble_the_product(sp, world, fmt):
    from paper_1805_11938_gb300.distributed import RowPartitioned

    a = synth.with_integer_values(synth.powerlaw(30_000, 21, xmax=2000, lmax=2000), 22)
    x = synth.integers(a.n, 23, -9, 9)
    xd = torch.as_tensor(x).cuda()
    parts = [RowPartitioned(a, r, world, None, fmt=fmt) for r in range(world)]
    assert sum(p.rows for p in parts) == a.m
    y = torch.cat([p.run(xd) for p in parts]).cpu().numpy()
    assert np.array_equal(bits(y), bits(oracle.csr_spmv(a, x)))
    xr = synth.vector(a.n, 24)
    ar = synth.powerlaw(30_000, 21, xmax=2000, lmax=2000)
    parts = [RowPartitioned(ar, r, world, None, fmt=fmt) for r in range(world)]
    yr = torch.cat([p.run(torch.as_tensor(xr).cuda()) for p in parts]).cpu().numpy()
    ok, msg = within_bound(ar, xr, yr)
    assert ok, msg


def test_selector_picks_each_block_format(sp):
    """With a model, every rank selects its own block's format."""
    from paper_1805_11938_gb300.distributed import RowPartitioned

    a = synth.stencil(synth.STENCIL_27PT_3D, 40, 40, 40, 25)
    model = sp.Model.load(sp.MODEL_PATH)
    parts = [RowPartitioned(a, r, 2, None, model=model) for r in range(2)]
    x = synth.vector(a.n, 26)
    y = torch.cat([p.run(torch.as_tensor(x).cuda()) for p in parts]).cpu().numpy()
    ok, msg = within_bound(a, x, y)
    assert ok, msg
    assert all(0 <= p.fmt < 5 for p in parts)
