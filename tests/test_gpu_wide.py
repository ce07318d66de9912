"""The iteration kernel with its per-edge arrays in global memory (the wide-
edge mode, te_options.edge_mode), through the C-ABI.

On instances that also fit shared memory, the global mode must give the same
bits as the shared-memory mode: the loads of Eq. 9 are exact integer sums in
both, so the whole run (rates, prices, beta and alpha decisions, residuals)
is identical.  On instances with more edges than a CTA's shared memory holds
(about 10,770), te_create takes the global mode by itself, and the iterate
must match the FP64 oracle within the 1e-4 bar of the other parity tests.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-4


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


def _scaled(inst, name):
    # demands scaled to half the total capacity, as the generator does for
    # all pairs, so that capacities bind on the subset too
    D = inst.demand * (0.5 * inst.capacity.sum() / inst.demand.sum())
    return dataclasses.replace(inst, name=name, demand=D)


@pytest.fixture(scope="module")
def wide_11k():
    # 1000-node WAN, 5,713 links = 11,426 directed edges, all pairs, k = 2
    from paper_2605_01748_b300 import instances
    return instances.make_waxman("wide-11k", 1000, 5800, 2, seed=0, locality=instances.LARGE_LOCALITY)


@pytest.fixture(scope="module")
def wide_30k():
    # 3000-node WAN, 15,111 links = 30,222 directed edges; 60,000 of its
    # 9M ordered pairs (k = 1), demands rescaled to half the total capacity
    from paper_2605_01748_b300 import instances
    full = instances.make_waxman("wide-30k", 3000, 15000, 1, seed=1, locality=instances.LARGE_LOCALITY)
    rng = np.random.default_rng(0)
    sub = instances.subset(full, np.sort(rng.choice(full.n_demands, 60000, replace=False)))
    return _scaled(sub, "wide-30k-sub")


def _torus(n, n_local, n_far, seed=0):
    """n x n torus of links (node (i, j) = i*n + j; link i*n + j to the right
    neighbour, n*n + i*n + j to the one below; edge 2l runs right or down,
    2l + 1 back), E = 4 n^2 directed edges.  Demands between n_local pairs
    at most 4 rows and columns apart and n_far random pairs, each with two
    paths (along the row, then the column, and the other way round; one path
    when the pair shares a row or column), every move the shorter way round.
    Capacities on {100, 200, 400}, lognormal demands scaled so that the paths
    carry twice the capacity of the edges they use."""
    from paper_2605_01748_b300.instances import Instance
    rng = np.random.default_rng(seed)
    N, NL = n * n, 2 * n * n
    a = np.arange(N)
    right = (a // n) * n + (a % n + 1) % n
    down = ((a // n + 1) % n) * n + a % n
    lsrc = np.concatenate([a, a]).astype(np.int32)
    ldst = np.concatenate([right, down]).astype(np.int32)
    esrc = np.empty(2 * NL, np.int32)
    edst = np.empty(2 * NL, np.int32)
    esrc[0::2], edst[0::2] = lsrc, ldst
    esrc[1::2], edst[1::2] = ldst, lsrc
    cap = np.repeat(rng.choice([100.0, 200.0, 400.0], NL), 2)

    def steps(i, j, d, axis):
        # edge ids of |d| moves from (i, j) along the axis (0: along the row)
        out = []
        for _ in range(abs(d)):
            if axis == 0:
                if d > 0:
                    out.append(2 * (i * n + j)); j = (j + 1) % n
                else:
                    j = (j - 1) % n; out.append(2 * (i * n + j) + 1)
            else:
                if d > 0:
                    out.append(2 * (N + i * n + j)); i = (i + 1) % n
                else:
                    i = (i - 1) % n; out.append(2 * (N + i * n + j) + 1)
        return out, i, j

    def short(d):
        d %= n
        return d if d <= n // 2 else d - n

    pairs = set()
    while len(pairs) < n_local:
        s = int(rng.integers(N))
        di, dj = rng.integers(-4, 5, 2)
        if di or dj:
            pairs.add((s, ((s // n + di) % n) * n + (s % n + dj) % n))
    while len(pairs) < n_local + n_far:
        s, t = (int(v) for v in rng.integers(N, size=2))
        if s != t:
            pairs.add((s, t))
    dsrc, ddst, dpo, peo, pe = [], [], [0], [0], []
    for s, t in sorted(pairs):
        si, sj, ti, tj = s // n, s % n, t // n, t % n
        dI, dJ = short(ti - si), short(tj - sj)
        h1, i1, j1 = steps(si, sj, dJ, 0)
        v1, _, _ = steps(i1, j1, dI, 1)
        paths = [h1 + v1]
        if dI and dJ:
            v2, i2, j2 = steps(si, sj, dI, 1)
            h2, _, _ = steps(i2, j2, dJ, 0)
            paths.append(v2 + h2)
        for p in paths:
            pe.extend(p)
            peo.append(len(pe))
        dsrc.append(s)
        ddst.append(t)
        dpo.append(len(peo) - 1)
    pe = np.asarray(pe, np.int32)
    dpo, peo = np.asarray(dpo, np.int64), np.asarray(peo, np.int64)
    D = rng.lognormal(0.0, 1.0, len(dsrc))
    hops = np.add.reduceat(np.diff(peo), dpo[:-1]) / np.diff(dpo)
    used = np.unique(pe)
    D *= 2.0 * cap[used].sum() / float((D * hops).sum())
    return Instance(f"torus-{n}", N, esrc, edst, cap, np.asarray(dsrc, np.int32), np.asarray(ddst, np.int32),
                    D, dpo, peo, pe, {"family": "torus", "n": n})


@pytest.fixture(scope="module")
def torus_67k():
    # 130 x 130 torus: 67,600 directed edges, beyond 16-bit ids
    return _torus(130, 18000, 2000)


def _same_run(te, inst, iters, **kw):
    a = te.TE(inst, **kw)
    b = te.TE(inst, edge_mode=te.EDGES_GLOBAL, **kw)
    assert a.layout()["edges_global"] == 0 and b.layout()["edges_global"] == 1
    ra, rb = a.solve(iters), b.solve(iters)
    for k in ("iters", "total_iters", "r", "s", "beta", "alpha", "converged"):
        assert ra[k] == rb[k], (k, ra[k], rb[k])
    xa, xb = a.allocation(project=te.PROJECT_NONE), b.allocation(project=te.PROJECT_NONE)
    assert np.array_equal(xa, xb)
    assert np.array_equal(a.prices(), b.prices())
    assert np.array_equal(a.trace(), b.trace())
    # the feasibility steps and the gap read only the iterate and the prices
    for proj in (te.PROJECT_ALG2, te.PROJECT_SCALE):
        assert np.array_equal(a.allocation(project=proj), b.allocation(project=proj))
    assert a.gap(project=te.PROJECT_SCALE) == b.gap(project=te.PROJECT_SCALE)
    a.close()
    b.close()


def test_global_mode_bit_identical_tiny(te, tiny):
    _same_run(te, tiny, 3000)


def test_global_mode_bit_identical_medium(te, medium):
    _same_run(te, medium, 600)


@pytest.mark.parametrize("alpha", [0.0, 1.0, 2.0])
def test_wide_instance_fixed_schedule_parity(te, wide_11k, alpha):
    assert wide_11k.n_edges > 10770
    kw = dict(alpha_target=alpha, alpha_start=alpha, beta0=1.0, adapt_beta=0, continuation=0, gamma=-1.0)
    t = te.TE(wide_11k, **kw)
    assert t.layout()["edges_global"] == 1 and t.layout()["id_bytes"] == 2
    assert t.solve(40)["iters"] == 40
    s = O.OracleSolver(wide_11k, **kw)
    s.run(40)
    x, xr = t.allocation(project=te.PROJECT_NONE), s.allocation()
    assert _rel_inf(x, xr) <= TOL
    Sg, Sr = O.demand_totals(wide_11k, x), O.demand_totals(wide_11k, xr)
    assert (np.abs(Sg - Sr) / np.maximum(Sr, 1e-2 * Sr.max())).max() <= TOL
    assert _rel_inf(t.prices(), s.prices()) <= TOL
    t.close()


def test_wide_instance_parity_and_feasibility(te, wide_30k):
    assert wide_30k.n_edges > 30000
    kw = dict(alpha_target=1.0, alpha_start=1.0, beta0=1.0, adapt_beta=0, continuation=0, gamma=-1.0)
    t = te.TE(wide_30k, **kw)
    t.solve(40)
    s = O.OracleSolver(wide_30k, **kw)
    s.run(40)
    assert _rel_inf(t.allocation(project=te.PROJECT_NONE), s.allocation()) <= TOL
    assert _rel_inf(t.prices(), s.prices()) <= TOL
    t.close()
    # the default solve (balancing, continuation, stop rule), then both
    # feasibility steps on its iterate
    t = te.TE(wide_30k)
    t.solve(5000)
    x = t.allocation(project=te.PROJECT_NONE)
    for proj in (te.PROJECT_ALG2, te.PROJECT_SCALE):
        xp = t.allocation(project=proj).astype(np.float64)
        loads = O.edge_loads(wide_30k, xp)
        assert (xp >= 0).all() and (loads <= wide_30k.capacity * (1 + 1e-5)).all()
        assert (O.demand_totals(wide_30k, xp) <= wide_30k.demand * (1 + 1e-5)).all()
    xs = O.project_scale(wide_30k, x.astype(np.float64))
    assert _rel_inf(t.allocation(project=te.PROJECT_SCALE), xs) <= 1e-5
    t.close()


def test_global_mode_needs_deterministic_loads(te, tiny, wide_30k):
    # FP32 histograms (4 B per edge instead of 8) fit shared memory up to
    # about 16,100 edges; 30,222 do not, and the global mode has no FP32 form
    with pytest.raises(te.TEError) as ei:
        te.TE(wide_30k, deterministic=0)
    assert ei.value.status == te.TE_EUNSUPPORTED
    with pytest.raises(te.TEError) as ei:
        te.TE(tiny, deterministic=0, edge_mode=te.EDGES_GLOBAL)
    assert ei.value.status == te.TE_EUNSUPPORTED


def test_32bit_ids_layout_and_walks(te, torus_67k):
    # the generator's paths are walks of the topology (te_create checks them)
    assert torus_67k.n_edges == 67600
    t = te.TE(torus_67k)
    info = t.layout()
    assert info["id_bytes"] == 4 and info["edges_global"] == 1
    t.close()


@pytest.mark.parametrize("alpha", [0.0, 1.0, 2.0])
def test_32bit_ids_fixed_schedule_parity(te, torus_67k, alpha):
    kw = dict(alpha_target=alpha, alpha_start=alpha, beta0=1.0, adapt_beta=0, continuation=0, gamma=-1.0)
    t = te.TE(torus_67k, **kw)
    t.solve(40)
    s = O.OracleSolver(torus_67k, **kw)
    s.run(40)
    x, xr = t.allocation(project=te.PROJECT_NONE), s.allocation()
    assert _rel_inf(x, xr) <= TOL
    Sg, Sr = O.demand_totals(torus_67k, x), O.demand_totals(torus_67k, xr)
    assert (np.abs(Sg - Sr) / np.maximum(Sr, 1e-2 * Sr.max())).max() <= TOL
    assert _rel_inf(t.prices(), s.prices()) <= TOL
    t.close()


def test_32bit_ids_feasibility_gap_and_refusal(te, torus_67k):
    t = te.TE(torus_67k, alpha_target=1.0, alpha_start=1.0, continuation=0)
    t.solve(3000)
    x = t.allocation(project=te.PROJECT_NONE).astype(np.float64)
    for proj in (te.PROJECT_ALG2, te.PROJECT_SCALE):
        xp = t.allocation(project=proj).astype(np.float64)
        loads = O.edge_loads(torus_67k, xp)
        assert (xp >= 0).all() and (loads <= torus_67k.capacity * (1 + 1e-5)).all()
        assert (O.demand_totals(torus_67k, xp) <= torus_67k.demand * (1 + 1e-5)).all()
    xs = O.project_scale(torus_67k, x)
    assert _rel_inf(t.allocation(project=te.PROJECT_SCALE), xs) <= 1e-5
    g, pr, du = t.gap(project=te.PROJECT_SCALE)
    xsg = t.allocation(project=te.PROJECT_SCALE).astype(np.float64)
    go, pro, duo = O.gap(torus_67k, xsg, t.prices(), 1.0)
    assert abs(du - duo) <= 1e-7 * abs(duo)
    assert abs(pr - pro) <= 2.0 ** -21 * torus_67k.n_demands
    t.close()
    with pytest.raises(te.TEError) as ei:
        te.TE(torus_67k, deterministic=0)
    assert ei.value.status == te.TE_EUNSUPPORTED


def test_32bit_ids_gradient_matches_oracle(te, torus_67k):
    # the differentiated form (fixed schedule, caller units) through 40
    # iterations with checkpoints every 7, against the oracle's reverse pass
    inst = torus_67k
    K, b0 = 40, inst.n_paths ** 2 / (inst.nnz * inst.demand.sum())
    t = te.TE(inst, alpha_target=1.0, alpha_start=1.0, beta0=b0, adapt_beta=0, continuation=0, gamma=-1.0,
              scale_mode=2)
    J, gC, gD = t.gradient(K, 7)
    Jo, gCo, gDo = O.gradient(inst, 1.0, b0, K)
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    g, go = np.concatenate([gC, gD]), np.concatenate([gCo, gDo])
    assert np.max(np.abs(g - go)) <= 1e-3 * np.max(np.abs(go))
    t.close()


def test_wide_mode_streaming_and_warm_start(te, wide_11k):
    # capacity change then reset equals a fresh handle on the changed
    # instance, bit for bit, in the global mode; a warm start after a demand
    # change keeps the run identical to the shared-memory mode's
    rng = np.random.default_rng(7)
    C2 = wide_11k.capacity * rng.uniform(0.5, 1.5, wide_11k.n_edges)
    a = te.TE(wide_11k)
    a.solve(100)
    a.set_capacities(C2)
    a.reset()
    ra = a.solve(200)
    b = te.TE(dataclasses.replace(wide_11k, capacity=C2))
    rb = b.solve(200)
    assert ra == rb
    assert np.array_equal(a.allocation(project=te.PROJECT_NONE), b.allocation(project=te.PROJECT_NONE))
    D2 = wide_11k.demand * rng.uniform(0.8, 1.2, wide_11k.n_demands)
    b.set_demands(D2)
    rb2 = b.solve(200)
    a.close()
    b.close()
    # the same sequence on an instance small enough for both modes
    from paper_2605_01748_b300 import instances
    m = instances.make_medium()
    D3 = m.demand * np.random.default_rng(8).uniform(0.8, 1.2, m.n_demands)
    runs = []
    for mode in (te.EDGES_AUTO, te.EDGES_GLOBAL):
        t = te.TE(m, edge_mode=mode)
        t.solve(300)
        t.set_demands(D3)
        r = t.solve(300)
        runs.append((r, t.allocation(project=te.PROJECT_NONE), t.prices()))
        t.close()
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][2], runs[1][2])
    assert rb2["iters"] > 0


def _parallel_links(E, K, seed=1):
    # E parallel one-hop links from node 0 to node 1; K demands with 1-4
    # one-hop paths on random links, a few on the highest ids
    from paper_2605_01748_b300.instances import Instance
    rng = np.random.default_rng(seed)
    npaths = rng.integers(1, 5, K)
    dpo = np.concatenate([[0], np.cumsum(npaths)]).astype(np.int64)
    P = int(dpo[-1])
    pe = rng.integers(0, E, P).astype(np.int32)
    pe[:20] = E - 1 - np.arange(20)
    return Instance(f"parallel-{E}", 2, np.zeros(E, np.int32), np.ones(E, np.int32), rng.uniform(1.0, 2.0, E),
                    np.zeros(K, np.int32), np.ones(K, np.int32), rng.uniform(0.5, 3.0, K), dpo,
                    np.arange(P + 1, dtype=np.int64), pe, {})


def test_edge_count_limit_of_the_global_mode(te):
    # each CTA's slice of the prices sits in shared memory beside the
    # staging buffers: 450,000 edges run (oracle parity), 600,000 are refused
    ok = _parallel_links(450000, 400)
    kw = dict(alpha_target=1.0, alpha_start=1.0, beta0=1.0, adapt_beta=0, continuation=0, gamma=-1.0)
    t = te.TE(ok, **kw)
    assert t.layout()["id_bytes"] == 4 and t.layout()["edges_global"] == 1
    t.solve(20)
    s = O.OracleSolver(ok, **kw)
    s.run(20)
    assert _rel_inf(t.allocation(project=te.PROJECT_NONE), s.allocation()) <= TOL
    t.close()
    with pytest.raises(te.TEError) as ei:
        te.TE(_parallel_links(600000, 400), **kw)
    assert ei.value.status == te.TE_EUNSUPPORTED and "edges" in str(ei.value)
