"""Host-side bookkeeping of bench.py that its JSON line rests on: how many
library kernels a product and a batch replay launch (the gpu_launches claim)."""
import bench


def _info(fmt, aux, sell_c=0):
    return {"fmt": fmt, "aux": list(aux), "params": {"sell_C": sell_c}}


def test_batch_families_follow_the_library_grouping():
    sell32, sell64, sell128 = (_info(3, [5, 10, 3, 0], c) for c in (32, 64, 128))
    assert bench.batch_families([sell32] * 3) == {"sell32"}
    assert bench.batch_families([sell32, sell64, sell128]) == {"sell32", "sell64", "sell128"}
    # CSR with tiles, and CSR without nonzeros (zeroed with the plain formats)
    assert bench.batch_families([_info(0, [4, 0, 0, 0]), _info(0, [0, 0, 0, 0])]) == {"csr", "other"}
    # CSR on the lanes-per-row path (aux[1] = V) runs with the plain formats
    assert bench.batch_families([_info(0, [4, 4, 0, 0])]) == {"other"}
    # HYB: the ELL part with the plain formats, the tail in its own family only when it has rows
    assert bench.batch_families([_info(4, [2, 7, 3, 1]), _info(4, [2, 0, 3, 0])]) == {"other", "hyb_tail"}
    assert bench.batch_families([_info(4, [2, 0, 3, 0])]) == {"other"}
    assert bench.batch_families([_info(1, [3, 0, 0, 0]), _info(2, [5, 0, 0, 0])]) == {"other"}
    assert bench.batch_families([_info(3, [0, 0, 0, 0], 32)]) == set()


def test_launches_per_run():
    assert bench.launches_per_run(0, _info(0, [4, 0, 0, 0])) == 1
    assert bench.launches_per_run(1, _info(1, [0, 0, 0, 0])) == 0  # nothing to do: no tiles, no zero rows
    assert bench.launches_per_run(1, _info(1, [3, 0, 0, 0])) == 1
    assert bench.launches_per_run(2, _info(2, [5, 0, 0, 0])) == 1
    assert bench.launches_per_run(3, _info(3, [5, 10, 3, 0], 32)) == 1
    assert bench.launches_per_run(3, _info(3, [5, 10, 3, 3], 32)) == 3  # one per column panel
    assert bench.launches_per_run(4, _info(4, [2, 7, 3, 1])) == 2  # ELL part + tail
    assert bench.launches_per_run(4, _info(4, [2, 0, 3, 0])) == 1
