"""Pins of the FP64 oracle against things other than itself.

* per-demand x-block: a generic constrained minimiser (SciPy SLSQP) on the
  same convex subproblem, and the closed-form proportional-fairness root of
  Appendix B.2 on the oracle's active set;
* the per-edge collapse: the expanded iteration that stores every consensus
  copy y_{e,r} and dual u_{e,r} (Eqs. 5-7, 10, 13);
* the limit of the iteration: the alpha = 0 linear program, the max-min LP
  sequence and textbook progressive filling, closed forms on the parking-lot
  and single-link networks, and the duality gap for alpha = 1;
* invariants: non-negative prices, the residual-balancing rule (Eq. 17) as
  recorded in the trace.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

import refsolvers as R
from oracle import oracle as O


# --------------------------------------------------------------------------
# per-demand subproblem (Section 3.3 "Rate Updates", Appendix B.2)
# --------------------------------------------------------------------------

def _subproblem_objective(x, m, w, alpha):
    S = x.sum()
    if alpha == 1.0:
        U = math.log(S) if S > 0 else -1e300
    else:
        U = (S ** (1 - alpha) - 1) / (1 - alpha) if S > 0 else (-1.0 / (1 - alpha) if alpha < 1 else -1e300)
    return -U + float(np.sum((x - m) ** 2 / (2 * w)))


def _brute(m, w, D, alpha, rng):
    n = m.shape[0]
    best = None
    cons = [{"type": "ineq", "fun": lambda x: D - x.sum()}]
    for _ in range(6):
        x0 = rng.random(n) * D / n * 0.9 + 1e-6
        res = minimize(_subproblem_objective, x0, args=(m, w, alpha), method="SLSQP",
                       bounds=[(0, None)] * n, constraints=cons, options={"ftol": 1e-14, "maxiter": 2000})
        if best is None or res.fun < best.fun:
            best = res
    return best.x


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0, 2.0, 3.5])
def test_demand_solve_matches_generic_minimiser(alpha):
    rng = np.random.default_rng(7)
    for trial in range(25):
        n = int(rng.integers(1, 7))
        m = rng.normal(0.0, 0.3, n)
        w = 1.0 / (rng.uniform(0.5, 4.0) * rng.integers(1, 6, n))
        D = float(rng.uniform(0.05, 1.5))
        lam, x = O.demand_solve(m, w, D, alpha)
        xb = _brute(m, w, D, alpha, rng)
        fo = _subproblem_objective(x, m, w, alpha)
        fb = _subproblem_objective(xb, m, w, alpha)
        # the oracle is never worse than the generic minimiser, and the
        # minimiser is unique (strictly convex in x)
        assert fo <= fb + 1e-9 * max(1.0, abs(fb)), (trial, fo, fb)
        assert np.allclose(x, xb, atol=2e-5), (trial, x, xb)
        assert (x >= 0).all() and x.sum() <= D * (1 + 1e-12)


def test_demand_solve_kkt_and_quadratic_root():
    """Stationarity x_r = max(0, m_r + lambda w_r); lambda = U'(S) when the cap
    is slack and lambda <= U'(D) when it binds.  For alpha = 1 on the final
    active set, lambda is the positive root of h lambda^2 + a lambda - 1 = 0
    (the quadratic of Appendix B.2)."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        n = int(rng.integers(1, 17))
        m = rng.normal(0.0, 0.2, n)
        w = 1.0 / (rng.uniform(0.1, 10.0) * rng.integers(1, 9, n))
        D = float(rng.uniform(0.01, 2.0))
        alpha = float(rng.choice([0.0, 1.0, 2.0, 5.0]))
        lam, x = O.demand_solve(m, w, D, alpha)
        assert np.allclose(x, np.maximum(0.0, m + lam * w), rtol=0, atol=1e-14)
        S = x.sum()
        if alpha == 0.0:
            assert lam <= 1.0 + 1e-12
            if lam < 1.0 - 1e-12:
                assert abs(S - D) <= 1e-12 * max(1.0, D)
        elif abs(S - D) > 1e-9 * D:
            assert abs(lam - S ** (-alpha)) <= 1e-9 * lam
            if alpha == 1.0:
                act = m + lam * w > 0
                a, h = m[act].sum(), w[act].sum()
                lam_q = 2.0 / (a + math.sqrt(a * a + 4.0 * h))
                assert abs(lam - lam_q) <= 1e-10 * lam
        else:
            assert lam <= D ** (-alpha) * (1 + 1e-9)


# --------------------------------------------------------------------------
# collapse of the per-incidence iteration to per-edge prices
# --------------------------------------------------------------------------

@pytest.mark.parametrize("alpha,beta", [(0.0, 2.0), (1.0, 0.5), (2.0, 4.0)])
def test_collapse_matches_expanded_iteration(tiny, alpha, beta):
    iters = 60
    s = O.OracleSolver(tiny, alpha_target=alpha, alpha_start=alpha, beta0=beta, adapt_beta=False,
                       continuation=False, gamma=-1.0)
    s.run(iters)
    x_e, y_e, u_e = O.run_expanded(tiny, beta, alpha, iters, scale=s.scale)
    assert np.max(np.abs(s.x - x_e)) <= 1e-11 * max(1.0, np.max(np.abs(x_e)))
    # every consensus dual on an edge equals that edge's price; y = x - d
    plen = np.diff(tiny.path_edge_off)
    xr = np.repeat(s.x, plen)
    assert np.max(np.abs(u_e - s.u[tiny.path_edges])) <= 1e-11
    assert np.max(np.abs(y_e - (xr - s.d[tiny.path_edges]))) <= 1e-11


# --------------------------------------------------------------------------
# limits of the iteration
# --------------------------------------------------------------------------

def test_alpha0_reaches_lp_optimum(tiny):
    lp_val, _ = R.lp_max_flow(tiny)
    s = O.solve(tiny, max_iters=20000, alpha_target=0.0, gamma=1e-6)
    assert s.converged
    xp = O.project(tiny, s.allocation(), 0.0)
    val = xp.sum()
    assert val <= lp_val * (1 + 1e-9)
    assert (lp_val - val) / lp_val <= 1e-3
    g, pr, du = O.gap(tiny, xp, s.prices(), 0.0)
    assert g >= -1e-9 and g / lp_val <= 2e-3


def test_alpha1_duality_gap_closes(tiny):
    s = O.solve(tiny, max_iters=50000, alpha_target=1.0, alpha_start=1.0, gamma=1e-7)
    assert s.converged
    xp = O.project(tiny, s.allocation(), 1.0)
    g, pr, du = O.gap(tiny, xp, s.prices(), 1.0)
    assert 0.0 <= g <= 1e-5 * abs(pr), (g, pr)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0, 4.0])
def test_parking_lot_closed_form(alpha):
    L = 3
    inst = R.parking_lot(L)
    s = O.solve(inst, max_iters=200000, alpha_target=alpha, alpha_start=alpha, gamma=1e-9)
    assert s.converged
    x = s.allocation()
    want = R.parking_lot_alpha_fair(L, alpha)
    assert abs(x[0] - want) <= 1e-5, (x[0], want)
    assert np.allclose(x[1:], 1.0 - want, atol=1e-5)


def test_parking_lot_alpha0_starves_long_flow():
    inst = R.parking_lot(3)
    s = O.solve(inst, max_iters=100000, alpha_target=0.0, gamma=1e-9)
    x = s.allocation()
    assert x[0] <= 1e-4 and np.allclose(x[1:], 1.0, atol=1e-4)


@pytest.mark.parametrize("alpha", [1.0, 3.0])
def test_single_link_water_filling(alpha):
    D = np.array([0.05, 0.1, 0.3, 0.4, 0.6, 0.9])
    inst = R.single_link(D, 1.0)
    s = O.solve(inst, max_iters=200000, alpha_target=alpha, alpha_start=alpha, gamma=1e-9)
    assert s.converged
    assert np.allclose(s.allocation(), R.water_level(D, 1.0), atol=1e-5)


def test_max_min_continuation_tiny(tiny):
    opt = R.lp_max_min(tiny)
    theta = 1e-6 * tiny.capacity.max()
    s = O.OracleSolver(tiny, alpha_target=math.inf, gamma=1e-3)
    best = 0.0
    while s.alpha < 3.0 and s.iters < 4000:
        s.run(25)
        xp = O.project(tiny, s.allocation(), s.alpha)
        best = max(best, O.optimality(O.demand_totals(tiny, xp), opt, theta))
    assert s.alpha >= 3.0
    assert best >= 0.99
    # alpha = 0 alone is clearly short of max-min on this instance
    s0 = O.solve(tiny, max_iters=5000, alpha_target=0.0)
    x0 = O.project(tiny, s0.allocation(), 0.0)
    assert O.optimality(O.demand_totals(tiny, x0), opt, theta) < 0.9


def test_max_min_single_path_matches_progressive_filling(tiny):
    k1 = R.first_path_only(tiny)
    pf = R.progressive_filling(k1)
    assert np.allclose(pf, R.lp_max_min(k1), rtol=1e-8, atol=1e-8)
    theta = 1e-6 * tiny.capacity.max()
    s = O.OracleSolver(k1, alpha_target=math.inf, gamma=1e-4)
    best = 0.0
    while s.iters < 6000 and s.alpha < 8:
        s.run(50)
        xp = O.project(k1, s.allocation(), s.alpha)
        best = max(best, O.optimality(O.demand_totals(k1, xp), pf, theta))
    assert best >= 0.995


# --------------------------------------------------------------------------
# invariants of the iteration
# --------------------------------------------------------------------------

def test_iteration_invariants_and_balancing_rule(tiny):
    s = O.OracleSolver(tiny, alpha_target=math.inf, gamma=1e-3)
    beta_prev = s.beta
    for _ in range(30):
        s.run(10)
        assert (s.u >= 0).all()
        assert (s.x >= 0).all()
    tr = s.trace
    beta_before = np.concatenate([[beta_prev], tr[:-1, 2]])
    r, sres, beta = tr[:, 0], tr[:, 1], tr[:, 2]
    up = r > 10 * sres
    down = (~up) & (sres > 10 * r)
    assert np.allclose(beta[up], 2 * beta_before[up])
    assert np.allclose(beta[down], beta_before[down] / 2)
    keep = ~(up | down)
    assert np.allclose(beta[keep], beta_before[keep])
    assert up.any() and keep.any()
    del beta_prev


def test_thread_count_does_not_change_results(tiny):
    a = O.solve(tiny, max_iters=120, alpha_target=math.inf, threads=1)
    b = O.solve(tiny, max_iters=120, alpha_target=math.inf, threads=4)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.u, b.u)


def test_exact_single_path_max_min_matches_progressive_filling(tiny):
    """The oracle's event-driven water-filling against the textbook
    progressive filling (rounds of equal increments) on single-path demands."""
    inst = R.first_path_only(tiny)
    a = O.maxmin_single_path(inst)
    b = R.progressive_filling(inst)
    assert np.max(np.abs(a - b) / np.maximum(b, 1e-12)) <= 1e-12


def test_exact_single_path_max_min_is_max_min(medium):
    """Feasible, and every demand is either at its cap or crosses a full
    edge on which no demand has a larger rate (the max-min certificate)."""
    inst = R.first_path_only(medium)
    a = O.maxmin_single_path(inst)
    L = O.edge_loads(inst, a)
    assert (L <= inst.capacity * (1 + 1e-12)).all()
    assert (a <= inst.demand * (1 + 1e-12)).all()
    full = L >= inst.capacity * (1 - 1e-9)
    emax = np.zeros(inst.n_edges)
    np.maximum.at(emax, inst.path_edges, a[np.repeat(np.arange(inst.n_demands), np.diff(inst.path_edge_off))])
    for c in range(inst.n_demands):
        if a[c] >= inst.demand[c] * (1 - 1e-12):
            continue
        es = inst.path_edges[inst.path_edge_off[c]:inst.path_edge_off[c + 1]]
        assert any(full[e] and a[c] >= emax[e] * (1 - 1e-9) for e in es), c


def test_printed_rate_suggestion_does_not_see_capacity(tiny):
    """The reading of the update equations: the rate suggestion as printed
    (Section 3.3, the cost of Eq. "penalty-b" and the suggestion built from
    its mean over the edge) subtracts from each path's cost the mean over
    the edge, so every term that is the same for all paths of the edge --
    the capacity and the capacity dual among them -- cancels.  Evaluating
    the printed formula for two capacities gives the same suggestions; the
    paper-literal multi-block variant would not enforce capacity, which is
    why the two-block reading (the capacity projection in the edge block)
    is implemented instead."""
    rng = np.random.default_rng(0)
    n = 7
    x = rng.uniform(0, 5, n)
    dual_con = rng.uniform(0, 1, n)
    beta = 0.7

    def printed(C, dual_cap):
        cost = beta * (-C - x) - dual_cap - dual_con
        return np.maximum((cost.mean() - cost) / beta, 0.0)

    assert np.allclose(printed(1.0, 0.3), printed(100.0, 7.0), rtol=0, atol=1e-12)


def test_oracle_structs_match_ctypes_mirrors():
    """The ctypes mirrors of the oracle's option and scalar structs have the
    C layout: every field set from Python comes back unchanged."""
    import ctypes
    lib = O._L()
    lib.or_echo_options.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.or_echo_scalars.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    vals = [1.5, 2.5, 3.5, 4.5, 5.5, 6.5, 7.5, 8.5, 9.5, 10.5, 11.5, 12, 13, 14, 15]
    o = O._Opts(*vals)
    out = np.zeros(16)
    lib.or_echo_options(ctypes.byref(o), out.ctypes.data)
    assert out[:15].tolist() == vals and out[15] == ctypes.sizeof(O._Opts)
    sc = O._Scalars(1.25, 2.25, 3.25, 4.25, 7, 8, 1, 0)
    out = np.zeros(8)
    lib.or_echo_scalars(ctypes.byref(sc), out.ctypes.data)
    assert out[:7].tolist() == [1.25, 2.25, 3.25, 4.25, 7, 8, 1] and out[7] == ctypes.sizeof(O._Scalars)


def test_max_norm_primal_residual_bounds_overload_at_stop(tiny):
    """With gamma_max set, a level counts as converged only when the largest
    n_e |u_e' - u_e| / C_e is within gamma_max.  An edge loaded above its
    capacity keeps a positive price, so its n_e (u_e' - u_e) is exactly
    L_e - C_e: at the stop every relative overload, recomputed here from the
    final rates, is within gamma_max (and the plain stop rule alone does not
    guarantee that)."""
    for gmax in (1e-2, 1e-3):
        s = O.OracleSolver(tiny, alpha_max=8.0, gamma_max=gmax)
        s.run(200000)
        assert s.converged
        over = (O.edge_loads(tiny, s.allocation()) - tiny.capacity) / tiny.capacity
        assert over.max() <= gmax * (1 + 1e-9), (gmax, over.max())
