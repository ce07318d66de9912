"""In-place updates of demands and capacities (streaming re-solve, warm
start): te_set_capacities / te_set_demands followed by te_reset reproduce a
handle built from the new inputs, a failed link (capacity 0) ends with no
load, and a warm re-solve after a demand change matches the oracle run on
the new demands from the same warm state."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_01748_b300.instances import Instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    from paper_2605_01748_b300 import build
    build.build_te()
    from paper_2605_01748_b300 import te as te_mod
    return te_mod


def _with(inst, capacity=None, demand=None):
    return Instance(inst.name, inst.n_nodes, inst.edge_src, inst.edge_dst,
                    inst.capacity if capacity is None else capacity, inst.demand_src, inst.demand_dst,
                    inst.demand if demand is None else demand, inst.demand_path_off, inst.path_edge_off,
                    inst.path_edges, dict(inst.meta))


def test_set_capacities_then_reset_matches_fresh_handle(te, medium):
    rng = np.random.default_rng(7)
    C2 = medium.capacity * rng.uniform(0.5, 1.5, medium.n_edges)
    a = te.TE(medium)
    a.solve(100)
    a.set_capacities(C2)
    a.reset()
    ra = a.solve(300)
    b = te.TE(_with(medium, capacity=C2))
    rb = b.solve(300)
    assert ra == rb
    xa, xb = a.allocation(project=te.PROJECT_NONE), b.allocation(project=te.PROJECT_NONE)
    assert np.array_equal(xa.view(np.uint32), xb.view(np.uint32))
    a.close()
    b.close()


def test_failed_link_carries_no_load(te, tiny):
    # the busiest edge of the initial allocation fails
    npaths = np.diff(tiny.demand_path_off)
    x0 = np.repeat(tiny.demand / npaths, npaths)
    e = int(np.argmax(O.edge_loads(tiny, x0)))
    C2 = tiny.capacity.copy()
    C2[e] = 0.0
    t = te.TE(tiny, gamma=1e-5)
    t.solve(500)
    t.set_capacities(C2)
    t.solve(20000)
    for mode in (te.PROJECT_ALG2, te.PROJECT_SCALE):
        xp = t.allocation(project=mode).astype(np.float64)
        L = O.edge_loads(tiny, xp)
        assert L[e] == 0.0
        assert (L <= C2 * (1 + 1e-5)).all()
    # every demand still reaches a positive rate over its other paths where it has one
    pe = tiny.path_edges
    peo = tiny.path_edge_off
    free = np.array([e not in pe[peo[r]:peo[r + 1]] for r in range(tiny.n_paths)])
    S = O.demand_totals(tiny, t.allocation(project=te.PROJECT_SCALE).astype(np.float64))
    has_free = np.add.reduceat(free.astype(int), tiny.demand_path_off[:-1]) > 0
    assert (S[has_free] > 0).all()
    t.close()


def test_warm_resolve_after_demand_change_matches_oracle(te, tiny):
    # unit max_e C_e (scale_mode 0): the capacities do not change, so both
    # sides normalise the new demands by the same unit
    kw = dict(alpha_target=1.0, alpha_start=1.0, beta0=1.0, adapt_beta=0, continuation=0, gamma=-1.0,
              scale_mode=0)
    t = te.TE(tiny, **kw)
    t.solve(200)
    x_mid = t.allocation(project=te.PROJECT_NONE)
    rng = np.random.default_rng(3)
    D2 = tiny.demand * np.exp(rng.uniform(np.log(0.8), np.log(1.2), tiny.n_demands))
    # the oracle restarts from the GPU's rates with zero prices: do the same
    t.set_demands(D2)
    t.warm_start(x_mid, keep_duals=False)
    t.solve(150)
    xg = t.allocation(project=te.PROJECT_NONE)
    s = O.OracleSolver(_with(tiny, demand=D2), x0=x_mid.astype(np.float64), **kw)
    s.run(150)
    xo = s.allocation()
    assert np.max(np.abs(xg - xo)) <= 1e-4 * np.max(np.abs(xo))
    t.close()
