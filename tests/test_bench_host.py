"""Host-side logic of bench.py (no GPU): the algorithmic byte count, the rule
that reports recorded DRAM traffic only for the captured kernel and
workload, the single-path variant and the command-line defaults."""
import json
import sys

import numpy as np
import pytest

import bench


def test_method_bytes_counts_each_unit(tiny):
    # 4 B per incidence, 12 B per path, 8 B per demand, 8 B per edge per CTA
    grid = 3
    by_hand = 0
    by_hand += 4 * int(tiny.path_edge_off[-1])
    by_hand += 12 * (len(tiny.path_edge_off) - 1)
    by_hand += 8 * len(tiny.demand)
    by_hand += 8 * grid * len(tiny.capacity)
    assert bench.method_bytes(tiny, grid) == by_hand
    # one more CTA adds one partial load per edge
    assert bench.method_bytes(tiny, grid + 1) - bench.method_bytes(tiny, grid) == 8 * len(tiny.capacity)


def test_kernel_hash_is_stable_and_short():
    h = bench.kernel_hash()
    assert h == bench.kernel_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)


@pytest.mark.parametrize("case", ["match", "other_workload", "other_sources", "missing"])
def test_traffic_reported_only_for_the_captured_kernel(tmp_path, monkeypatch, case):
    rec = {"workload": "large", "kernel_source_sha256_16": bench.kernel_hash(), "dram_bytes_per_iteration": 123456789}
    if case == "other_sources":
        rec["kernel_source_sha256_16"] = "0" * 16
    path = tmp_path / "traffic.json"
    if case != "missing":
        path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "NCU_TRAFFIC_JSON", str(path))
    value, why = bench.ncu_traffic("medium" if case == "other_workload" else "large")
    if case == "match":
        assert value == 123456789.0
    else:
        assert value is None and why


def test_recorded_traffic_file_is_well_formed():
    rec = json.load(open(bench.NCU_TRAFFIC_JSON))
    assert rec["workload"] in ("tiny", "medium", "large")
    assert rec["dram_bytes_per_iteration"] > 0
    assert len(rec["kernel_source_sha256_16"]) == 16
    assert "--clock-control none" in rec["command"]


def test_first_path_variant_keeps_each_demands_first_path(tiny):
    v = bench.first_path_variant(tiny)
    n = len(tiny.demand)
    assert len(v.demand) == n
    assert np.array_equal(v.demand_path_off, np.arange(n + 1))
    for c in range(n):
        r = tiny.demand_path_off[c]
        a, b = tiny.path_edge_off[r], tiny.path_edge_off[r + 1]
        a1, b1 = v.path_edge_off[c], v.path_edge_off[c + 1]
        assert np.array_equal(v.path_edges[a1:b1], tiny.path_edges[a:b])
    assert v.meta["k"] == 1


def test_defaults_time_the_large_workload(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.workload == "large" and a.impl == "ours"
    assert a.warmup >= 3 and a.steps >= 1
    assert a.feasibility == 0 and a.steady == "" and a.iters == 0
