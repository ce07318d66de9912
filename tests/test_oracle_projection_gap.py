"""Pins of the oracle's feasibility projection (Algorithm 2) and duality gap.

Projection: post-conditions of Theorem 1(A) (x >= 0, S_c <= D_c, L_e <= C_e),
identity on feasible inputs, and a hand-worked example whose trimming order
is fixed by the scores.  Gap: weak duality on random feasible points and
prices, and tightness at the alpha = 0 LP optimum with the LP's own
capacity multipliers (strong duality, Slater point of Appendix C).
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import refsolvers as R
from oracle import oracle as O
from paper_2605_01748_b300.instances import Instance


def _perturbed(inst, rng, scale=0.4):
    """A random, clearly infeasible allocation: demands spread over paths and
    inflated, some entries negative."""
    npaths = np.diff(inst.demand_path_off)
    base = np.repeat(inst.demand / npaths, npaths)
    return base * rng.uniform(0.2, 2.5, base.shape[0]) - scale * base * (rng.random(base.shape[0]) < 0.1)


@pytest.mark.parametrize("alpha", [0.0, 1.0, 3.0])
def test_projection_postconditions(tiny, alpha):
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = _perturbed(tiny, rng)
        xp = O.project(tiny, x, alpha)
        assert (xp >= 0).all()
        assert (O.demand_totals(tiny, xp) <= tiny.demand * (1 + 1e-12)).all()
        assert (O.edge_loads(tiny, xp) <= tiny.capacity * (1 + 1e-12)).all()
        # trimming only: no path gains rate beyond max(x, 0)
        assert (xp <= np.maximum(x, 0) + 1e-12).all()


def test_projection_keeps_feasible_points(tiny):
    rng = np.random.default_rng(5)
    x = O.project(tiny, _perturbed(tiny, rng), 1.0)
    # edges trimmed to exactly C_e may read a rounding-level excess when
    # their load is re-summed; nothing beyond that may change
    assert np.allclose(O.project(tiny, x, 1.0), x, rtol=0, atol=1e-12)


def _two_demand_example():
    """Hand-worked case.  Edges: e0 (C=1), e1 (C=10), e2 (C=10).
    Demand A (D=2) has paths a0 = [e0], a1 = [e1, e0], a2 = [e2].
    Demand B (D=5) has path b0 = [e0, e1].
    x = (a0, a1, a2, b0) = (1.0, 0.5, 1.0, 0.75).
      S_A = 2.5 > D_A = 2 -> E_A = 0.5;  L_e0 = 2.25 > 1 -> V_e0 = 1.25.
      C_p: a0 = 1, a1 = 1, a2 = 0, b0 = 1 (only e0 is violated).
      Demand step (alpha = 1): scores S_A * C_p tie for a0 and a1 (2.5),
      lower index first -> a0 loses 0.5: x = (0.5, 0.5, 1.0, 0.75).
      Recompute: S_A = 2, S_B = 0.75, L_e0 = 1.75 -> V_e0 = 0.75.
      Edge step on e0: scores a0 = a1 = 2 * 1, b0 = 0.75 * 1.
      Order a0, a1, b0: a0 trimmed by 0.5, a1 by 0.25.
      Result x = (0.0, 0.25, 1.0, 0.75)."""
    cap = np.array([1.0, 10.0, 10.0])
    inst = Instance("hand", 3, np.array([0, 0, 0], np.int32), np.array([1, 1, 1], np.int32), cap,
                    np.array([0, 0], np.int32), np.array([1, 1], np.int32), np.array([2.0, 5.0]),
                    np.array([0, 3, 4], np.int64), np.array([0, 1, 3, 4, 6], np.int64),
                    np.array([0, 1, 0, 2, 0, 1], np.int32), {})
    x = np.array([1.0, 0.5, 1.0, 0.75])
    return inst, x, np.array([0.0, 0.25, 1.0, 0.75])


def test_projection_hand_example():
    inst, x, want = _two_demand_example()
    assert np.allclose(O.project(inst, x, 1.0), want, atol=1e-15)


def test_projection_edge_step_uses_largest_planned_trim():
    """Two violated edges plan different trims for a shared path; the path
    loses the larger one and both edges end feasible.
    Edges e0 (C=1), e1 (C=1).  Paths: p0 = [e0, e1] (demand 0), p1 = [e0]
    (demand 1), p2 = [e1] (demand 2); x = (1, 0.5, 0.2), alpha = 0 so the
    score is the violation count: p0 has 2, p1 and p2 have 1.
    e0: V = 0.5, first p0 -> plan 0.5.   e1: V = 0.2, first p0 -> plan 0.2.
    p0 loses max(0.5, 0.2) = 0.5 -> x = (0.5, 0.5, 0.2)."""
    inst = Instance("two-edges", 3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.ones(2),
                    np.array([0, 0, 1], np.int32), np.array([2, 1, 2], np.int32), np.array([5.0, 5.0, 5.0]),
                    np.arange(4, dtype=np.int64), np.array([0, 2, 3, 4], np.int64),
                    np.array([0, 1, 0, 1], np.int32), {})
    xp = O.project(inst, np.array([1.0, 0.5, 0.2]), 0.0)
    assert np.allclose(xp, [0.5, 0.5, 0.2], atol=1e-15)


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0, 2.0])
def test_gap_weak_duality(tiny, alpha):
    rng = np.random.default_rng(9)
    for _ in range(10):
        x = O.project(tiny, _perturbed(tiny, rng), alpha)
        p = rng.exponential(0.01, tiny.n_edges) * (rng.random(tiny.n_edges) < 0.7)
        if alpha > 0:
            p = p * np.mean(tiny.demand) ** (-alpha)
        g, pr, du = O.gap(tiny, x, p, alpha)
        assert g >= -1e-9 * max(1.0, abs(pr)), (g, pr, du)


def test_gap_tight_at_lp_optimum(tiny):
    AE, AD = R._incidence(tiny)
    A = sp.vstack([AE, AD]).tocsr()
    b = np.concatenate([tiny.capacity, tiny.demand])
    res = linprog(-np.ones(tiny.n_paths), A_ub=A, b_ub=b, bounds=(0, None), method="highs")
    x = res.x
    p = -res.ineqlin.marginals[:tiny.n_edges]
    g, pr, du = O.gap(tiny, x, p, 0.0)
    assert abs(g) <= 1e-7 * abs(pr)
    # a wrong price (all zero) must show a large gap
    g0, _, _ = O.gap(tiny, x, np.zeros(tiny.n_edges), 0.0)
    assert g0 > 1e-2 * abs(pr)


# ---------------- proportional feasibility scaling (not in the paper) ----------------

def test_project_scale_postconditions(tiny):
    rng = np.random.default_rng(11)
    for _ in range(5):
        x = _perturbed(tiny, rng)
        xp = O.project_scale(tiny, x)
        assert (xp >= 0).all()
        assert (O.demand_totals(tiny, xp) <= tiny.demand * (1 + 1e-12)).all()
        assert (O.edge_loads(tiny, xp) <= tiny.capacity * (1 + 1e-12)).all()
        # scaling only: every path keeps a fraction in (0, 1] of max(x, 0)
        xc = np.maximum(x, 0)
        assert (xp <= xc * (1 + 1e-15)).all()
        assert ((xp > 0) == (xc > 0)).all()


def test_project_scale_keeps_feasible_points(tiny):
    rng = np.random.default_rng(13)
    x = O.project_scale(tiny, _perturbed(tiny, rng))
    x = x * (1 - 1e-9)  # strictly inside: no factor may fire
    assert np.array_equal(O.project_scale(tiny, x), x)


def test_project_scale_hand_example():
    """Same instance as the Algorithm 2 example, x = (1, 0.5, 1, 0.75).
    Demand A: S_A = 2.5 > 2 -> factor 0.8: (a0, a1, a2) = (0.8, 0.4, 0.8).
    Loads: e0 = a0 + a1 + b0 = 1.95 > 1 -> f_e0 = 1/1.95; e1 = a1 + b0 =
    1.15 <= 10; e2 = a2 = 0.8 <= 10.  Paths through e0 (a0, a1, b0) are
    scaled by 1/1.95, a2 is kept: x = (0.8, 0.4, 0.8*1.95, 0.75) / 1.95."""
    inst, x, _ = _two_demand_example()
    want = np.array([0.8 / 1.95, 0.4 / 1.95, 0.8, 0.75 / 1.95])
    got = O.project_scale(inst, x)
    assert np.allclose(got, want, rtol=1e-15, atol=0)
    assert abs(O.edge_loads(inst, got)[0] - 1.0) <= 1e-15


def test_project_scale_uses_smallest_edge_factor():
    """A path on two violated edges takes the smaller factor of the two.
    Edges e0 (C=1), e1 (C=1); p0 = [e0, e1], p1 = [e0], p2 = [e1];
    x = (1, 1, 3): L_e0 = 2 -> 1/2, L_e1 = 4 -> 1/4.  p0 -> 1/4, p1 -> 1/2,
    p2 -> 3/4; loads end at e0 = 0.75, e1 = 1."""
    inst = Instance("two-edges", 3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.ones(2),
                    np.array([0, 0, 1], np.int32), np.array([2, 1, 2], np.int32), np.array([5.0, 5.0, 5.0]),
                    np.arange(4, dtype=np.int64), np.array([0, 2, 3, 4], np.int64),
                    np.array([0, 1, 0, 1], np.int32), {})
    xp = O.project_scale(inst, np.array([1.0, 1.0, 3.0]))
    assert np.allclose(xp, [0.25, 0.5, 0.75], rtol=0, atol=1e-15)
