"""Host logic of bench.py's roofline line (no GPU): the byte and draw models
of each sampler kind, and the measured-traffic figure, which is reported only
for the kernel source it was taken on."""
import os
import sys
from types import SimpleNamespace

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _result(**kw):
    base = dict(draws=0, cta_draws=0, edge_visits=0, cta_edge_visits=0, node_visits=0, cta_node_visits=0,
                n_rr=0, cta_sets=0, pool_entries=0, cta_stored_entries=0, cta_stored_sets=0,
                trace=[{"n_sets": 0}])
    base.update(kw)
    return SimpleNamespace(**base)


def test_gap_walk_roofline_is_hbm_bytes_per_visit():
    # warp class: 1000 visited nodes, 100 sets of which 80 stored with 900 entries, 500 draws
    r = _result(node_visits=1000, n_rr=100, pool_entries=900, trace=[{"n_sets": 80}], draws=500,
                edge_visits=123456)
    ks = {"sample_warp": {"launches": 2, "ms": 1.0}}
    roof = bench.roofline("ic_wc", "sample_warp", ks, [r], 152, 2070.0, "no-such-workload", 6789.6, "measured")
    # 16 per visit + 8 per live edge taken (visits - sets) + 8 per stored entry + 12 per stored set
    # + 1 per hit-tested set
    abytes = 16 * 1000 + 8 * (1000 - 100) + 8 * 900 + 12 * 80 + (100 - 80)
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(abytes / 2)
    assert roof["achieved"] == pytest.approx(abytes / 1e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6789.6)
    assert roof["traffic"] is None  # no capture for this workload


def test_edge_record_roofline_is_philox_issue():
    r = _result(node_visits=10, cta_node_visits=10, cta_draws=4000, draws=4000, cta_edge_visits=16000,
                edge_visits=16000, n_rr=3, cta_sets=3)
    ks = {"sample_cta": {"launches": 1, "ms": 2.0}}
    roof = bench.roofline("ic_records", "sample_cta", ks, [r], 152, 2070.0, "x", 6789.6, "measured")
    peak = 152 * 4 * 2070e6 * 32 / bench.PHILOX_MIN_INSTR
    assert roof["bound"] == "alu" and roof["peak"] == pytest.approx(peak)
    assert roof["achieved"] == pytest.approx(4000 / 2e-3)


def test_traffic_only_for_the_captured_source(monkeypatch):
    r = _result(node_visits=1000, n_rr=10, pool_entries=1000, trace=[{"n_sets": 10}])
    ks = {"sample_warp": {"launches": 4, "ms": 1.0}}
    key = ("w", "sample_warp")
    monkeypatch.setitem(bench.TRAFFIC, key, {"src": bench.kernel_source_hash(), "bytes_per_node_visit": 300.0})
    roof = bench.roofline("ic_wc", "sample_warp", ks, [r], 152, 2070.0, "w", 6789.6, "measured")
    assert roof["traffic"] == pytest.approx(300.0 * 1000 / 4)
    assert roof["traffic_gbs"] == pytest.approx(300.0 * 1000 / 4 / (1.0 / 4 / 1000.0) / 1e9)
    monkeypatch.setitem(bench.TRAFFIC, key, {"src": "0000000000000000", "bytes_per_node_visit": 300.0})
    roof = bench.roofline("ic_wc", "sample_warp", ks, [r], 152, 2070.0, "w", 6789.6, "measured")
    assert roof["traffic"] is None


def test_no_roofline_outside_the_samplers():
    ks = {"greedy": {"launches": 1, "ms": 5.0}}
    assert bench.roofline("ic_wc", "greedy", ks, [_result()], 152, 2070.0, "w", 6789.6, "measured") is None
    assert bench.roofline("lt", "sample_warp", {"sample_warp": {"launches": 1, "ms": 1.0}}, [_result()], 152,
                          2070.0, "w", 6789.6, "measured") is None


def test_recorded_traffic_matches_this_source():
    # the committed traffic figures were taken on the committed sampler source
    for (workload, cls), tr in bench.TRAFFIC.items():
        assert tr["src"] == bench.kernel_source_hash(), (workload, cls)
