"""The committed ncu summaries bench.py reads its roofline traffic from: each carries
a parseable traffic record (bytes per launch, the kernel sources and their hash at
capture time), and bench.py reports the figure only while the sources are unchanged."""
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("name", ["multigrid_cycle_beam_lognormal_1024_dt50.md",
                                  "step_traffic_beam_lognormal_1024_dt50.md",
                                  "step_traffic_gas_point_source_256.md"])
def test_traffic_record_parses(name):
    import bench
    from paper_2011_13926_gb300.ncu_summary import source_hash
    traffic, rec = bench.profile_traffic(name)
    assert rec["status"] in ("current", "stale: the kernel sources changed since the capture"), rec
    assert rec["source_sha_now"] != "" and len(rec["source_sha_at_capture"]) == 16
    if rec["status"] == "current":
        assert traffic > 0.0
    else:
        assert traffic is None


def test_missing_profile_is_reported():
    import bench
    traffic, rec = bench.profile_traffic("no_such_profile.md")
    assert traffic is None and rec["status"] == "missing"


def test_mg_cycle_bytes_by_hand():
    """bytes_mg_cycle at 1024^2 with 7 levels, term by term (FP32 words, n_u = 3, d = 2)."""
    import bench
    lv = [1024 ** 2, 512 ** 2, 256 ** 2, 128 ** 2, 64 ** 2, 32 ** 2, 16 ** 2]
    nu, jv_in = 3, 3 + 1 + 2
    w = lv[0] * ((nu + 9 + nu + jv_in) + (nu + nu + jv_in + 9 + nu)) + 2 * nu * lv[1]
    for l in range(1, 6):
        w += lv[l] * ((45 + 9 + 2 * nu) + (45 + 9 + 3 * nu)) + 2 * nu * lv[l + 1]
    w += lv[6] * (45 + 9 + 2 * nu)
    assert bench.bytes_mg_cycle(1024, 1024, 7) == 4 * w
    assert bench.bytes_jv32(1024 ** 2) == 48 * 1024 ** 2  # the scope table's 48 B per cell (2D, FP32)


def test_complete_units_keeps_whole_cycles():
    """A capture cut off by its launch count keeps whole units only: from the first
    unit start through the last unit end (a multigrid cycle runs from the level-0 down
    pass to the level-0 up pass)."""
    from paper_2011_13926_gb300.ncu_summary import complete_units, summarise
    m = {"dram__bytes_read.sum": 10.0, "dram__bytes_write.sum": 0.0, "gpu__time_duration.sum": 1e-6}
    seq = ["jv", "down0", "mg", "up0", "jv", "down0", "mg", "up0", "jv", "down0", "mg"]
    launches = [(str(i), n, dict(m)) for i, n in enumerate(seq)]
    kept = complete_units(launches, "down0", "up0")
    assert [n for _, n, _ in kept] == seq[1:8]
    _, traffic, units = summarise(kept, select="down0|mg|up0", units_regex="down0")
    assert units == 2 and traffic == 30.0  # three launches of 10 bytes per whole cycle
    assert complete_units(launches, "nothing", "up0") == []
