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
file measures that on the tiny instance and records the numbers; it needs
no GPU.  Test infrastructure only."""
import numpy as np

from oracle import oracle as O


def _literal_run(inst, alpha, beta, iters):
    """The printed multi-block iteration; returns the path rates (caller units)."""
    scale = float(np.exp(np.mean(np.log(inst.demand))))
    C = inst.capacity / scale
    D = inst.demand / scale
    P, K = inst.n_paths, inst.n_demands
    plen = np.diff(inst.path_edge_off)
    inc_path = np.repeat(np.arange(P), plen)          # path of each incidence
    inc_edge = inst.path_edges.astype(np.int64)       # edge of each incidence
    path_dem = np.repeat(np.arange(K), np.diff(inst.demand_path_off))
    n_e = np.bincount(inc_edge, minlength=inst.n_edges).astype(np.float64)
    x = np.repeat(D / np.diff(inst.demand_path_off), np.diff(inst.demand_path_off))
    y = x[inc_path].copy()
    d_dem = np.zeros(K)
    d_cap = np.zeros(inst.n_edges)
    d_con = np.zeros(inc_edge.shape[0])
    d_neg = np.zeros(P)
    w = 1.0 / (1.0 + plen)
    for _ in range(iters):
        S = np.bincount(path_dem, weights=x, minlength=K)
        # dual updates from x^k, y^k
        d_dem_n = np.maximum(d_dem + (S - D), 0.0)
        d_cap_n = np.maximum(d_cap + (np.bincount(inc_edge, weights=y, minlength=inst.n_edges) - C), 0.0)
        d_con_n = np.maximum(d_con + (x[inc_path] - y), 0.0)
        d_neg_n = np.maximum(d_neg - x, 0.0)
        # rate suggestions
        cost = beta * (-C[inc_edge] - x[inc_path]) - d_cap_n[inc_edge] - d_con_n
        mean_e = np.bincount(inc_edge, weights=cost, minlength=inst.n_edges) / np.maximum(n_e, 1.0)
        y_n = np.maximum((mean_e[inc_edge] - cost) / beta, 0.0)
        # rate computation from the previous y and duals
        Q = np.bincount(inc_path, weights=y - d_con, minlength=P)
        a = np.bincount(path_dem, weights=w * (Q + d_neg), minlength=K)
        W = np.bincount(path_dem, weights=w, minlength=K)
        # S (1 + W) = a + W (D - d_dem) + W S^-alpha / beta, solved by bisection (the
        # right side falls as S grows for alpha > 0; alpha = 0 is linear)
        rhs0 = a + W * (D - d_dem)
        if alpha == 0.0:
            S_new = (rhs0 + W / beta) / (1.0 + W)
        else:
            lo = np.full(K, 1e-12)
            hi = np.maximum(1.0, np.abs(rhs0) + W / beta) * 10.0 + 1.0
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                f = mid * (1.0 + W) - rhs0 - W * mid ** (-alpha) / beta
                lo = np.where(f < 0, mid, lo)
                hi = np.where(f < 0, hi, mid)
            S_new = 0.5 * (lo + hi)
        Sp = S_new[path_dem]
        x = w * (Q + Sp ** (-alpha) / beta - (Sp - D[path_dem] + d_dem[path_dem]) + d_neg) if alpha > 0.0 else \
            w * (Q + 1.0 / beta - (Sp - D[path_dem] + d_dem[path_dem]) + d_neg)
        y, d_dem, d_cap, d_con, d_neg = y_n, d_dem_n, d_cap_n, d_con_n, d_neg_n
    return x * scale


def _violation(inst, x):
    L = O.edge_loads(inst, np.maximum(x, 0.0))
    return float(np.max((L - inst.capacity) / inst.capacity))


def test_printed_multiblock_iteration_does_not_enforce_capacity(tiny):
    """After 2000 iterations at alpha = 1 the printed iteration leaves edges
    far over capacity, while the two-block reading (the oracle) meets the
    capacities to within its stop tolerance."""
    x_lit = _literal_run(tiny, alpha=1.0, beta=1.0, iters=2000)
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
    x1 = _literal_run(tiny, alpha=1.0, beta=1.0, iters=300)
    x2 = _literal_run(dataclasses.replace(tiny, capacity=2.0 * tiny.capacity), alpha=1.0, beta=1.0, iters=300)
    assert np.allclose(x1, x2, rtol=1e-12, atol=1e-12)
