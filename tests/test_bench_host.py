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
    assert bench.launches_per_run(3, _info(3, [5, 10, 3, -1], 32)) == 1  # rows in place: one kernel too
    assert bench.launches_per_run(3, _info(3, [5, 10, 3, 3], 32)) == 4  # one per column panel, one unpermuting y
    assert bench.launches_per_run(4, _info(4, [2, 7, 3, 1])) == 2  # ELL part + tail
    assert bench.launches_per_run(4, _info(4, [2, 0, 3, 0])) == 1


def test_algorithmic_bytes_closed_forms():
    """Every stored nonzero once (12 B), x (8N) and y (8M) once, plus each format's
    metadata, never the padding."""
    m, n, nnz = 1000, 700, 5000
    base = 12 * nnz + 8 * n + 8 * m

    def info(aux):
        return {"m": m, "n": n, "nnz": nnz, "aux": list(aux), "params": {"sell_C": 32}}

    assert bench.algorithmic_bytes(0, info([15, 0, 0, 0])) == base + 4 * (m + 1)     # CSR: ptr
    assert bench.algorithmic_bytes(1, info([5, 0, 0, 0])) == base + 5 * 160          # CSR5: 160 B per tile
    assert bench.algorithmic_bytes(2, info([7, 0, 0, 0])) == base + 4 * m            # ELL: row_len
    assert bench.algorithmic_bytes(3, info([32, 40, 9, 0])) == base + 8 * m + 8 * 33 + 8 * 40  # SELL
    # SELL whose sort moved no row (aux[3] = -1): row_len only, perm is not read
    assert bench.algorithmic_bytes(3, info([32, 40, 9, -1])) == base + 4 * m + 8 * 33 + 8 * 40
    assert bench.algorithmic_bytes(4, info([2, 30, 3, 1])) == base + 4 * m + 16 * 30  # HYB: 16 B per tail row
    # the padding a layout stores does not count: the same matrix in ELL moves the same nonzeros
    assert bench.algorithmic_bytes(2, info([7000, 0, 0, 0])) == bench.algorithmic_bytes(2, info([7, 0, 0, 0]))


def test_clock_sampler_summary():
    """nvidia-smi lines (no GPU needed): median SM clock, maximum clock, and the throttle
    reasons seen active in any sample; malformed lines are skipped."""
    cs = bench.ClockSampler(0)
    cs.f.write("0, 2070, 2070, 812.3, 0x0, Not Active, Not Active, Not Active, Not Active\n"
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
               "garbage line\n"
               "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs2 = bench.ClockSampler(0)
    cs2.f.write("0, 1000, 2070, 500, 0x8, Active, Not Active, Active, Not Active\n")
    assert cs2.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                                               "samples": 0}


def test_traffic_counts_only_for_the_captured_parameters(tmp_path, monkeypatch):
    """An ncu traffic figure recorded with the captured launch's tuning
    parameters is reported only for a handle resolved to the same ones."""
    import json

    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({
        "w:SELL": [{"bytes": 10, "params": {"sell_C": 64, "sell_sigma": 1}},
                   {"bytes": 20, "params": {"sell_C": 64, "sell_sigma": 500}}],
        "w:CSR5": {"bytes": 30, "params": {"csr5_sigma": 32}},
        "w:CSR": 40}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("w:SELL", {"sell_C": 64, "sell_sigma": 1, "hyb_k": 0}) == 10
    assert bench.load_traffic("w:SELL", {"sell_C": 64, "sell_sigma": 500}) == 20
    assert bench.load_traffic("w:SELL", {"sell_C": 32, "sell_sigma": 1}) is None
    assert bench.load_traffic("w:CSR5", {"csr5_sigma": 24}) is None
    assert bench.load_traffic("w:CSR5", {"csr5_sigma": 32}) == 30
    assert bench.load_traffic("w:CSR", {}) == 40
    assert bench.load_traffic("w:ELL", {}) is None
