"""The batch engine (one instance per CTA, one launch for many what-if
instances) against the FP64 oracle run on each instance alone, and against
the single-instance engine."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_01748_b300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    from paper_2605_01748_b300 import build
    build.build_te()
    from paper_2605_01748_b300 import te as te_mod
    return te_mod


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))


def test_batch_matches_oracle_per_instance(te, tiny):
    W = instances.make_what_if(tiny, 3, 2, seed=2, min_fail=1, max_fail=1)
    kw = dict(alpha_target=1.0, alpha_start=1.0, beta0=1.0, adapt_beta=0, continuation=0, gamma=-1.0)
    b = te.TEBatch(W, **kw)
    res = b.solve(150)
    assert all(r["iters"] == 150 for r in res)
    for i, inst in enumerate(W):
        s = O.OracleSolver(inst, **kw)
        s.run(150)
        assert _rel(b.allocation(i, project=te.PROJECT_NONE), s.allocation()) <= 1e-4
    info = b.info()
    # six instances: te_solve's iteration kernel with SMs / 6 CTAs each
    assert info["n_instances"] == 6 and info["ctas_per_instance"] >= 2 and info["warps_per_cta"] == 20
    b.close()


def test_batch_kernel_one_instance_per_cta_matches_oracle(te, tiny):
    """More instances than half the SMs: the batch kernel (one instance per
    CTA, CUDA graph, autotuned CTA shape) against the oracle per instance."""
    W = instances.make_what_if(tiny, 40, 2, seed=6, min_fail=1, max_fail=2)
    kw = dict(alpha_target=1.0, alpha_start=1.0, beta0=1.0, adapt_beta=0, continuation=0, gamma=-1.0)
    b = te.TEBatch(W, **kw)
    res = b.solve(120)
    info = b.info()
    assert info["n_instances"] == 80 and info["ctas_per_instance"] == 0 and info["warps_per_cta"] in (8, 16)
    assert all(r["iters"] == 120 for r in res)
    for i in (0, 37, 79):
        s = O.OracleSolver(W[i], **kw)
        s.run(120)
        assert _rel(b.allocation(i, project=te.PROJECT_NONE), s.allocation()) <= 1e-4
    b.close()


def test_grouped_batch_matches_single_engine_bit_for_bit(te, medium):
    """The grouped launch runs te_solve's own iteration kernel on fewer CTAs
    per instance; the edge loads are exact integer sums, so after a fixed
    schedule the rates equal the single engine's bit for bit."""
    W = instances.make_what_if(medium, 2, 1, seed=8)
    kw = dict(alpha_target=2.0, alpha_start=2.0, beta0=1.0, adapt_beta=0, continuation=0, gamma=-1.0)
    b = te.TEBatch(W, **kw)
    assert b.info()["ctas_per_instance"] >= 2
    b.solve(50)
    for i, inst in enumerate(W):
        t = te.TE(inst, **kw)
        t.solve(50)
        xs = t.allocation(project=te.PROJECT_NONE)
        xb = b.allocation(i, project=te.PROJECT_NONE)
        assert np.array_equal(xs.view(np.uint32), xb.view(np.uint32))
        t.close()
    b.close()


def test_batch_matches_single_engine_with_adaptive_beta(te, medium):
    W = instances.make_what_if(medium, 2, 2, seed=3)
    b = te.TEBatch(W)
    res = b.solve(300)
    for i, inst in enumerate(W):
        t = te.TE(inst)
        r = t.solve(300)
        assert (r["total_iters"], r["alpha"], r["beta"]) == (res[i]["total_iters"], res[i]["alpha"], res[i]["beta"])
        xs = t.allocation(project=te.PROJECT_NONE)
        assert _rel(b.allocation(i, project=te.PROJECT_NONE), xs) <= 1e-5
        t.close()
    b.close()


def test_batch_projection_matches_oracle_per_instance(te, tiny):
    """Algorithm 2 on each instance of a batch (one list of violated
    incidences for all instances, grown when an instance needs more) against
    the oracle's projection of that instance's iterate."""
    W = instances.make_what_if(tiny, 4, 2, seed=3, min_fail=1, max_fail=2)
    b = te.TEBatch(W, gamma=-1.0)
    b.solve(20)
    res = b.solve(0)
    trimmed = 0
    for i, inst in enumerate(W):
        x = b.allocation(i, project=te.PROJECT_NONE).astype(np.float64)
        xg = b.allocation(i, project=te.PROJECT_ALG2)
        xo = O.project(inst, x, res[i]["alpha"])
        assert _rel(xg, xo) <= 1e-4, (i, _rel(xg, xo))
        assert (O.edge_loads(inst, xg) <= inst.capacity * (1 + 1e-5) + 1e-9).all()
        trimmed += int((xg < x.astype(np.float32)).any())
    assert trimmed > 0  # the iterates had violations to trim
    b.close()


def test_batch_stops_each_instance_by_its_own_rule(te, tiny):
    W = instances.make_what_if(tiny, 4, 1, seed=4)
    b = te.TEBatch(W, gamma=1e-3)
    res = b.solve(50000)
    for i, inst in enumerate(W):
        assert res[i]["converged"] == 1
        t = te.TE(inst, gamma=1e-3)
        r = t.solve(50000)
        assert r["converged"] == 1
        assert abs(r["total_iters"] - res[i]["total_iters"]) <= max(5, 0.02 * r["total_iters"])
        for mode in (te.PROJECT_ALG2, te.PROJECT_SCALE):
            xp = b.allocation(i, project=mode).astype(np.float64)
            assert (O.edge_loads(inst, xp) <= inst.capacity * (1 + 1e-5) + 1e-9).all()
            assert (O.demand_totals(inst, xp) <= inst.demand * (1 + 1e-5)).all()
        t.close()
    # a second call with no budget left changes nothing
    res2 = b.solve(0)
    assert [r["total_iters"] for r in res2] == [r["total_iters"] for r in res]
    b.close()
