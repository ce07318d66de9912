"""NEXT-4 as a measured ablation: the update equations as printed (Section
3.3), run as a multi-block iteration on the 12-node instance, against the
two-block reading that the library implements.

The printed iteration (Algorithm 1's order; all in normalised units, the
consensus duals per incidence):
  dual_dem  <- [dual_dem + (S(x) - D)]_+                       (dual-updates-dem)
  dual_cap  <- [dual_cap + (sum_r y_{e,r} - C_e)]_+            (dual-updates-cap)
  dual_con  <- [dual_con + (x_r - y_{e,r})]_+                  (dual-updates-con)
  dual_neg  <- [dual_neg - x_r]_+                              (dual-updates-neg)
  cost_{e,r} = beta (-C_e - x_r) - dual_cap_e - dual_con_{e,r} (penalty-b)
  y_{e,r}   <- [(mean_e cost - cost_{e,r}) / beta]_+           (rate-suggestion)
  x_r       <- (Q_r + S^-alpha / beta - (S - D + dual_dem) + dual_neg_r) / (1 + n_r),
               Q_r = sum_{e in r} (y_{e,r} - dual_con_{e,r}), with S the demand's
               total, found from the sum of that formula over its paths
                                                                (rate-computation)
where the rate formula takes the previous y and duals (the rate equation's
superscripts).  The capacity and its dual are the same for every path of an
edge, so they cancel in the rate suggestion: nothing in the iteration sees
C_e, and the loads settle where the demands and the utility put them.  This
file pins the oracle's restatement (oracle.literal_run) on two iterations
worked by hand, and measures the capacity effect on the tiny instance; it
needs no GPU."""
import numpy as np

from oracle import oracle as O


def test_two_iterations_worked_by_hand():
    """One demand D = 2 on one one-hop path over a link of capacity C = 1,
    alpha = 0, beta = 1.  Normalised by the geometric mean of the demands
    (2): D = 1, C = 0.5, x0 = y0 = 1, duals 0.
    Iteration 1: S = 1, dual_dem = 0, dual_cap = [1 - 0.5]_+ = 0.5,
    dual_con = [1 - 1]_+ = 0, dual_neg = 0; the only incidence's cost is its
    edge's mean, so y = 0.  Rate from the previous y and duals: Q = 1,
    w = 1/2, a = w Q = 1/2, W = 1/2, rhs0 = a + W (D - 0) = 1, S = (rhs0 +
    W / beta) / (1 + W) = 1, x = w (Q + 1 - (S - D) + 0) = 1.
    Iteration 2: S = 1, dual_dem = 0, dual_cap = [0.5 + 0 - 0.5]_+ = 0,
    dual_con = [0 + 1 - 0]_+ = 1, dual_neg = 0, y = 0.  Rate: Q = y - dual_con
    (both previous) = 0, a = 0, rhs0 = 1/2, S = (1/2 + 1/2) / (3/2) = 2/3,
    x = (1/2)(0 + 1 - (2/3 - 1) + 0) = 2/3, i.e. 4/3 in caller units."""
    import refsolvers as R
    inst = R.single_link(np.array([2.0]), 1.0)
    assert np.allclose(O.literal_run(inst, alpha=0.0, beta=1.0, iters=1), [2.0], rtol=0, atol=1e-15)
    assert np.allclose(O.literal_run(inst, alpha=0.0, beta=1.0, iters=2), [4.0 / 3.0], rtol=0, atol=1e-15)


def _violation(inst, x):
    L = O.edge_loads(inst, np.maximum(x, 0.0))
    return float(np.max((L - inst.capacity) / inst.capacity))


def test_printed_multiblock_iteration_does_not_enforce_capacity(tiny):
    """After 2000 iterations at alpha = 1 the printed iteration leaves edges
    far over capacity, while the two-block reading (the oracle) meets the
    capacities to within its stop tolerance."""
    x_lit = O.literal_run(tiny, alpha=1.0, beta=1.0, iters=2000)
    v_lit = _violation(tiny, x_lit)
    s = O.OracleSolver(tiny, alpha_target=1.0, alpha_start=1.0, gamma=1e-6)
    s.run(20000)
    v_two = _violation(tiny, s.allocation())
    # measured: the printed iteration overloads the busiest edge by a factor
    # of several; the two-block iterate is within 1e-4 of feasibility
    assert v_lit > 0.5, v_lit
    assert v_two < 1e-3, v_two


def test_printed_iteration_ignores_capacity_values(tiny):
    """The same run with every capacity doubled gives the same rates: the
    capacities never enter the printed iteration's rates."""
    import dataclasses
    x1 = O.literal_run(tiny, alpha=1.0, beta=1.0, iters=300)
    x2 = O.literal_run(dataclasses.replace(tiny, capacity=2.0 * tiny.capacity), alpha=1.0, beta=1.0, iters=300)
    assert np.allclose(x1, x2, rtol=1e-12, atol=1e-12)
