"""The host-side measurement logic of bench.py, on CPU: the algorithmic bytes of a query, the
expansion budget, the L calibration with its interpolation at recall 0.90, the traffic-record
lookup and the clock summary.  The search itself is faked (recall as a function of L)."""
import math
import types

import pytest

import bench


def test_method_bytes_per_query_c2():
    # id-1M-768, d = 160 LVQ-8: query 3072 B, a graph row 4 R + 4 = 260 B, a primary record
    # 160 + 8 -> 192 B (32-byte sectors), a secondary record 768 + 8 = 776 B
    assert bench.method_bytes_per_query(768, 160, 8, 64, hops=1, scored=0, rerank=0) == 3072 + 260
    assert bench.method_bytes_per_query(768, 160, 8, 64, hops=0, scored=1, rerank=0) == 3072 + 192
    assert bench.method_bytes_per_query(768, 160, 8, 64, hops=0, scored=0, rerank=1) == 3072 + 776
    # LVQ-4 primaries of d = 160: 80 code bytes + 8 -> 96 B
    assert bench.method_bytes_per_query(768, 160, 4, 64, hops=0, scored=1, rerank=0) == 3072 + 96
    # the benchmark's operating point: 76 hops, 879.3 scored, 152 reranked -> 309.6 KB
    b = bench.method_bytes_per_query(768, 160, 8, 64, 76.0, 879.3195, 152)
    assert b == pytest.approx(3072 + 76 * 260 + 879.3195 * 192 + 152 * 776)
    assert round(b / 1000, 1) == 309.6


def test_hop_limit():
    assert bench.hop_limit(0.0, 152) == 0
    assert bench.hop_limit(0.5, 152) == 76
    assert bench.hop_limit(0.5, 151) == 76  # ceil
    assert bench.hop_limit(1.33, 36) == 48
    assert bench.hop_limit(1.0, 128) == 128


def _fake_recall(monkeypatch, slope):
    monkeypatch.setattr(bench, "recall_at", lambda ids, truth, k: min(1.0, 0.5 + ids / slope))


def test_calibrate_smallest_grid_L(monkeypatch):
    _fake_recall(monkeypatch, 310.0)  # recall 0.90 at L = 124: the grid's 128 is the first at or above
    L, trace = bench.calibrate(lambda L: L, None, 10)
    assert L == 128
    assert trace[-1][0] == 128 and trace[-1][1] >= 0.90 and trace[-2][1] < 0.90
    _fake_recall(monkeypatch, 1e9)  # never reaches 0.90
    L, trace = bench.calibrate(lambda L: L, None, 10)
    assert L is None and len(trace) == len(bench.L_GRID)


def test_calibrate_budget_interpolates_in_log_qps(monkeypatch):
    _fake_recall(monkeypatch, 310.0)
    qps = {}

    def time_fn(L, mh):
        qps[(L, mh)] = 1e9 / L
        return qps[(L, mh)]

    L, mh, rec, table = bench.calibrate_budget(lambda L, mh: L, time_fn, None, 10, factors=(0.5, 1.0))
    assert L == 128 and mh in (64, 128)
    row = [t for t in table if t["hop_factor"] == 0.5][0]
    (L0, r0), (L1, r1) = row["recall_trace"]
    assert (L0, L1) == (120, 128)
    assert row["qps"] == pytest.approx(1e9 / 128) and row["qps_below"] == pytest.approx(1e9 / 120)
    f = (0.90 - r0) / (r1 - r0)
    want = math.exp(math.log(1e9 / 120) + f * (math.log(1e9 / 128) - math.log(1e9 / 120)))
    assert row["qps_interpolated"] == pytest.approx(want)
    # between the two grid points' QPS, and the grid value is the one reported
    assert row["qps"] < row["qps_interpolated"] < row["qps_below"]


def test_calibrate_budget_first_grid_point_reaches_target(monkeypatch):
    _fake_recall(monkeypatch, 20.0)  # recall 1.0 at the grid's first L: no point below to interpolate
    L, mh, rec, table = bench.calibrate_budget(lambda L, mh: L, lambda L, mh: 5.0, None, 10, factors=(0.5,))
    assert L == bench.L_GRID[0]
    assert table[0]["qps_interpolated"] == 5.0 and "qps_below" not in table[0]


def test_recorded_traffic_keys():
    a = types.SimpleNamespace(n=1_000_000, m=10_000, width=2, hash=0, projection="bf16", alpha=1.02, rule=1,
                              graph="full", secondary="lvq8", vbits=0)
    sha = bench.beam_src_sha1()
    rec = [r for r in bench.TRAFFIC_RECORDS if r["src_sha1"] == sha]
    got = bench.recorded_traffic(a, 152, 76)
    if not rec:  # the search sources changed since the last capture: no traffic is claimed
        assert got is None
        return
    want = [r["bytes"] for r in rec if r["L"] == 152 and r.get("max_hops") == 76 and r.get("vbits", 32) == 32]
    assert got == (want[0] if want else None)
    # any other configuration, or another slot width without its own capture, has none
    assert bench.recorded_traffic(a, 148, 76) is None
    a.width = 1
    assert bench.recorded_traffic(a, 152, 76) is None


def test_clock_summary():
    c = bench.Clocks(0)
    c.lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_best_hop_factor_and_shared_config():
    table = [{"hop_factor": 0.0, "L": None}, {"hop_factor": 0.5, "L": 152, "qps": 8.8e6},
             {"hop_factor": 0.6, "L": 140, "qps": 8.6e6}]
    assert bench.best_hop_factor(table, 1.0) == 0.5
    assert bench.best_hop_factor([{"hop_factor": 0.5, "L": None}], 1.0) == 1.0
    args = types.SimpleNamespace(n=1_000_000, D=768, d=160, R=64, L_build=128, alpha=1.02, rule=1, graph="full",
                                 secondary="lvq8", projection="bf16", hash=0, width=2, qpw=0, vbits=0)
    inf = {"primary_stride": 192, "secondary_stride": 800, "R": 64}
    c = bench.id_config(args, "id-1000k-768", 10_000, 152, 76, 0.5, inf)
    # what is searched and how, no results: the same dict in the benchmark's and the reference's line
    assert c["L"] == c["rerank"] == 152 and c["max_hops"] == 76 and c["width"] == 2
    assert not any(k in c for k in ("recall_at_10", "hop_budget_table", "build_seconds", "impl_note"))
    assert c["l2"].startswith("inputs larger than L2 (index 1.25 GB")
