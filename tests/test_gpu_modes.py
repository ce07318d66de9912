"""Options of the C-ABI on the GPU: the non-deterministic load accumulation
(te_options.deterministic = 0) against the FP64 oracle, and te_solve's
per-call tolerance (the gamma of Eq. 18 for one call)."""
import math

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the same bar as the deterministic path (tests/test_gpu_parity.py)


@pytest.fixture(scope="module")
def te():
    from paper_2605_01748_b300 import build
    build.build_te()
    from paper_2605_01748_b300 import te as te_mod
    return te_mod


def _rel_inf(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _check(inst, xg, xo):
    assert _rel_inf(xg, xo) <= TOL, _rel_inf(xg, xo)
    Sg, So = O.demand_totals(inst, xg), O.demand_totals(inst, xo)
    err = np.abs(Sg - So) / np.maximum(So, 1e-2 * So.max())
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("alpha,beta0", [(0.0, 2.0), (1.0, 1.0), (2.0, 4.0)])
def test_fp32_atomic_loads_parity_tiny(te, tiny, alpha, beta0):
    """One FP32 shared-memory add per incidence: the loads differ from the
    exact sums only by FP32 rounding, so the 1e-4 parity still holds."""
    kw = dict(alpha_target=alpha, alpha_start=alpha, beta0=beta0, adapt_beta=0, continuation=0, gamma=-1.0)
    t = te.TE(tiny, deterministic=0, **kw)
    assert t.solve(60)["iters"] == 60
    s = O.OracleSolver(tiny, **kw)
    s.run(60)
    _check(tiny, t.allocation(project=False), s.allocation())
    assert _rel_inf(t.prices(), s.prices()) <= TOL
    t.close()


def test_fp32_atomic_loads_parity_medium(te, medium):
    kw = dict(alpha_target=1.0, alpha_start=1.0, beta0=2.0, adapt_beta=0, continuation=0, gamma=-1.0)
    t = te.TE(medium, deterministic=0, **kw)
    t.solve(40)
    s = O.OracleSolver(medium, **kw)
    s.run(40)
    _check(medium, t.allocation(project=False), s.allocation())
    t.close()


def test_fp32_atomic_loads_adaptive_medium(te, medium):
    """Default options: the residuals of the two modes agree closely over the
    first iterations (the beta schedule only differs once a residual ratio
    sits within rounding of the balancing threshold)."""
    a = te.TE(medium)
    b = te.TE(medium, deterministic=0)
    a.solve(200)
    b.solve(200)
    ta, tb = a.trace(200), b.trace(200)
    diff = np.where(ta[:, 2] != tb[:, 2])[0]
    first = int(diff[0]) if diff.size else 200
    assert first >= 50, first
    np.testing.assert_allclose(ta[:first, :2], tb[:first, :2], rtol=1e-3, atol=1e-7)
    a.close()
    b.close()


def test_per_call_tolerance_matches_oracle_gamma(te, tiny):
    """te_solve(tol) uses tol as gamma for that call: the run stops exactly
    where the oracle created with gamma = tol stops."""
    t = te.TE(tiny)
    r = t.solve(20000, 1e-2)
    s = O.OracleSolver(tiny, gamma=1e-2)
    s.run(20000)
    assert r["converged"] == 1 and s.converged
    assert r["iters"] == s.iters
    assert r["alpha"] == s.alpha
    # a later call without tol runs on with te_options.gamma (1e-3)
    r2 = t.solve(1)
    assert r2["iters"] == 1
    t.close()


def test_zero_tolerance_runs_all_iterations(te, tiny):
    t = te.TE(tiny, alpha_target=1.0, alpha_start=1.0)
    r = t.solve(500, 0.0)
    assert r["iters"] == 500 and r["converged"] == 0
    t.close()


def test_nan_tolerance_rejected(te, tiny):
    t = te.TE(tiny)
    with pytest.raises(te.TEError) as ei:
        t.solve(10, math.nan)
    assert ei.value.status == te.TE_EINVAL
    t.close()


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_beta_bound_matches_oracle(te, tiny, medium, name):
    """With beta_max the balancing never raises beta above beta_max * beta0;
    the GPU and the oracle take the same beta and alpha decisions."""
    inst = tiny if name == "tiny" else medium
    iters = 1500 if name == "tiny" else 400
    t = te.TE(inst, beta_max=8.0)
    t.solve(iters)
    s = O.OracleSolver(inst, beta_max=8.0)
    s.run(iters)
    tg, to = t.trace(iters), s.trace
    n = min(tg.shape[0], to.shape[0])
    beta0 = s.sc.beta0  # the initial penalty (the same on both sides up to summation order)
    assert np.all(tg[:, 2] <= 8.0 * beta0 * (1 + 1e-9)) and np.all(to[:, 2] <= 8.0 * beta0 * (1 + 1e-12))
    diff = np.where((np.abs(tg[:n, 2] / to[:n, 2] - 1.0) > 1e-9) | (tg[:n, 3] != to[:n, 3]))[0]
    first = int(diff[0]) if diff.size else n
    assert first >= min(n, 100), first
    t.close()
