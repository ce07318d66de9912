"""Host-side logic of bench.py (no GPU): the algorithmic byte count, the rule
that reports recorded DRAM traffic only for the captured kernel and
workload, the single-path variant and the command-line defaults."""
import json
import math
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


def _u_hom(S, alpha):
    # the alpha-fair objective (Eq. 4) without its constant: sum log S at
    # alpha = 1, else sum S^(1-alpha) / (1-alpha), homogeneous in S
    S = np.asarray(S, dtype=np.float64)
    return float(np.sum(np.log(S))) if alpha == 1.0 else float(np.sum(S ** (1.0 - alpha)) / (1.0 - alpha))


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
def test_certificate_bounds_the_distance_to_the_exact_optimum(alpha):
    # one link: every alpha-fair optimum (alpha > 0) is water-filling, so U* is
    # known in closed form; at any iterate the certificate from the oracle's
    # gap must bound the true distance, and close once the iteration has
    from oracle import oracle as O
    import refsolvers as R
    D = np.array([0.05, 0.1, 0.3, 0.4, 0.6, 0.9]) * 10.0
    inst = R.single_link(D, 10.0)
    n = inst.n_demands
    u_star = _u_hom(R.water_level(D, 10.0), alpha)
    s = O.OracleSolver(inst, alpha_target=alpha, alpha_start=alpha, continuation=0, gamma=-1.0)
    seen = []
    for it in (3, 10, 30, 3000):
        s.run(it - s.iters)
        x = O.project_scale(inst, s.allocation())
        g, pr, du = O.gap(inst, x, s.prices(), alpha)
        u = _u_hom(x, alpha)  # one path per demand: S = x
        shift = 0.0 if alpha == 1.0 else n / (1.0 - alpha)
        assert pr + shift == pytest.approx(u, rel=1e-12, abs=1e-12)
        assert u <= u_star + 1e-12 * abs(u_star) and du + shift >= u_star - 1e-12 * abs(u_star)
        true = (u_star - u) / n if alpha == 1.0 else (u_star - u) / abs(u_star)
        eps = bench.certified_eps(g, pr, du, alpha, n)
        assert true <= eps + 1e-12
        seen.append(eps)
    assert seen[-1] <= 1e-6 and seen[0] > seen[-1]


def test_certificate_bounds_the_lp_distance_tiny(tiny):
    # alpha = 0 on the 12-node instance against the exact LP optimum
    from oracle import oracle as O
    import refsolvers as R
    lp, _ = R.lp_max_flow(tiny)
    n = tiny.n_demands
    s = O.OracleSolver(tiny, alpha_target=0.0, alpha_start=0.0, continuation=0, gamma=-1.0)
    for it in (20, 100):
        s.run(it - s.iters)
        x = O.project_scale(tiny, s.allocation())
        g, pr, du = O.gap(tiny, x, s.prices(), 0.0)
        thr = float(x.sum())
        assert pr + n == pytest.approx(thr, rel=1e-12)
        assert thr <= lp * (1 + 1e-9) and du + n >= lp * (1 - 1e-9)
        assert (lp - thr) / lp <= bench.certified_eps(g, pr, du, 0.0, n) + 1e-12


def test_certificate_edge_cases():
    n = 10
    assert bench.certified_eps(math.inf, -math.inf, 1.0, 1.0, n) == math.inf
    # alpha = 0: primal_h = primal + n
    assert bench.certified_eps(2.0, 0.0, 2.0, 0.0, n) == pytest.approx(0.2)
    # alpha = 2: primal_h = primal - n
    assert bench.certified_eps(2.0, -2.0, 0.0, 2.0, n) == pytest.approx(0.2)
    assert bench.certified_eps(5.0, -100.0, -95.0, 1.0, n) == pytest.approx(0.5)
    # a bracket through zero certifies nothing
    assert bench.certified_eps(1.0, -2.0, -1.0, 0.5, 1) == math.inf
