"""Exact reference solutions used to pin the oracle (test infrastructure).

None of these share code with the oracle or the CUDA path; they solve the TE
problem of GATE Section 3.1 (Eqs. 1-4) by independent textbook means:

* :func:`lp_max_flow` -- alpha = 0 (total throughput, Table 3) as one linear
  program (SciPy/HiGHS).
* :func:`lp_max_min` -- the max-min fair demand totals (alpha -> infinity,
  Table 3) by the standard sequence of linear programs: raise a common level
  for all unfrozen demands, then freeze every demand that cannot exceed it.
* :func:`progressive_filling` -- single-path max-min by textbook progressive
  filling (exact, event driven).
* Closed forms: the parking-lot network and the single shared link.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog

from paper_2605_01748_b300.instances import Instance


def _incidence(inst: Instance):
    """A_E [E x P] (path-edge) and A_D [K x P] (demand-path) 0/1 matrices."""
    P = inst.n_paths
    plen = np.diff(inst.path_edge_off)
    rows = inst.path_edges.astype(np.int64)
    cols = np.repeat(np.arange(P), plen)
    AE = sp.csr_matrix((np.ones(rows.shape[0]), (rows, cols)), shape=(inst.n_edges, P))
    npaths = np.diff(inst.demand_path_off)
    AD = sp.csr_matrix((np.ones(P), (np.repeat(np.arange(inst.n_demands), npaths), np.arange(P))),
                       shape=(inst.n_demands, P))
    return AE, AD


def lp_max_flow(inst: Instance):
    """max sum_r x_r s.t. A_E x <= C, A_D x <= D, x >= 0.  Returns (value, x)."""
    AE, AD = _incidence(inst)
    A = sp.vstack([AE, AD]).tocsr()
    b = np.concatenate([inst.capacity, inst.demand])
    res = linprog(-np.ones(inst.n_paths), A_ub=A, b_ub=b, bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    return -res.fun, res.x


def lp_max_min(inst: Instance):
    """Exact max-min fair demand totals S (unique) by progressive LPs.

    Each round maximises a common level t for the unfrozen demands (frozen
    ones keep their level).  By complementary slackness, a demand whose
    constraint S_c >= t has a positive multiplier in the optimal dual is at
    S_c = t in every optimal solution, so it is frozen at t; the multipliers
    sum to one, so every round freezes at least one demand."""
    AE, AD = _incidence(inst)
    K, P = inst.n_demands, inst.n_paths
    frozen = np.zeros(K, dtype=bool)
    level = np.zeros(K)
    while not frozen.all():
        free = np.where(~frozen)[0]
        fz = np.where(frozen)[0]
        nf = free.shape[0]
        A_rows = [sp.hstack([AE, sp.csr_matrix((inst.n_edges, 1))]),
                  sp.hstack([AD, sp.csr_matrix((K, 1))]),
                  sp.hstack([-AD[free], sp.csr_matrix(np.ones((nf, 1)))])]
        b_rows = [inst.capacity, inst.demand, np.zeros(nf)]
        if fz.size:
            A_rows.append(sp.hstack([-AD[fz], sp.csr_matrix((fz.size, 1))]))
            b_rows.append(-level[fz] * (1 - 1e-12))
        A = sp.vstack(A_rows).tocsr()
        b = np.concatenate(b_rows)
        c = np.zeros(P + 1)
        c[-1] = -1.0
        res = linprog(c, A_ub=A, b_ub=b, bounds=(0, None), method="highs")
        assert res.status == 0, res.message
        t = res.x[-1]
        off = inst.n_edges + K
        mult = -res.ineqlin.marginals[off:off + nf]
        block = mult > 1e-9
        block |= inst.demand[free] <= t * (1 + 1e-12)
        assert block.any(), "no demand froze: numerical trouble"
        newly = free[block]
        level[newly] = np.minimum(t, inst.demand[newly])
        frozen[newly] = True
    return level


def progressive_filling(inst: Instance) -> np.ndarray:
    """Max-min fair totals when every demand has exactly one path."""
    npaths = np.diff(inst.demand_path_off)
    assert (npaths == 1).all(), "progressive filling needs single-path demands"
    K = inst.n_demands
    edges_of = [inst.path_edges[inst.path_edge_off[c]:inst.path_edge_off[c + 1]] for c in range(K)]
    rate = np.zeros(K)
    active = np.ones(K, dtype=bool)
    residual = inst.capacity.astype(np.float64).copy()
    while active.any():
        cnt = np.zeros(inst.n_edges)
        for c in np.where(active)[0]:
            cnt[edges_of[c]] += 1
        with np.errstate(divide="ignore"):
            edge_inc = np.where(cnt > 0, residual / np.where(cnt > 0, cnt, 1), np.inf)
        dem_inc = np.where(active, inst.demand - rate, np.inf)
        inc = min(edge_inc.min(), dem_inc.min())
        rate[active] += inc
        for c in np.where(active)[0]:
            residual[edges_of[c]] -= inc
        sat = (cnt > 0) & (residual <= 1e-12 * inst.capacity)
        for c in np.where(active)[0]:
            if rate[c] >= inst.demand[c] * (1 - 1e-12) or sat[edges_of[c]].any():
                active[c] = False
    return rate


def first_path_only(inst: Instance) -> Instance:
    """The k = 1 variant of an instance: every demand keeps its first path."""
    first = inst.demand_path_off[:-1]
    plen = inst.path_edge_off[first + 1] - inst.path_edge_off[first]
    peo = np.concatenate([[0], np.cumsum(plen)]).astype(np.int64)
    pe = np.concatenate([inst.path_edges[inst.path_edge_off[r]:inst.path_edge_off[r + 1]] for r in first])
    return dataclasses.replace(inst, name=inst.name + "-k1", demand_path_off=np.arange(inst.n_demands + 1,
                               dtype=np.int64), path_edge_off=peo, path_edges=pe.astype(np.int32),
                               meta=dict(inst.meta, k=1))


def parking_lot(L: int, long_demand: float = 10.0, short_demand: float = 10.0) -> Instance:
    """A chain of L unit-capacity links; one demand spans all of them on a
    single path and L one-hop demands each use one link."""
    n = L + 1
    src = np.arange(L, dtype=np.int32)
    dst = np.arange(1, L + 1, dtype=np.int32)
    cap = np.ones(L)
    dsrc = np.concatenate([[0], np.arange(L)]).astype(np.int32)
    ddst = np.concatenate([[L], np.arange(1, L + 1)]).astype(np.int32)
    D = np.concatenate([[long_demand], np.full(L, short_demand)])
    dpo = np.arange(L + 2, dtype=np.int64)
    peo = np.concatenate([[0, L], L + np.arange(1, L + 1)]).astype(np.int64)
    pe = np.concatenate([np.arange(L), np.arange(L)]).astype(np.int32)
    return Instance("parking-lot", n, src, dst, cap, dsrc, ddst, D, dpo, peo, pe, {"L": L})


def parking_lot_alpha_fair(L: int, alpha: float) -> float:
    """alpha-fair rate of the long flow: U'(x) = L U'(1 - x), i.e.
    x = 1 / (1 + L^(1/alpha)) for alpha > 0 (demands not binding)."""
    return 1.0 / (1.0 + L ** (1.0 / alpha))


def single_link(demands: np.ndarray, capacity: float) -> Instance:
    """n single-path demands sharing one link."""
    n = demands.shape[0]
    return Instance("single-link", 2, np.array([0], np.int32), np.array([1], np.int32),
                    np.array([float(capacity)]), np.zeros(n, np.int32), np.ones(n, np.int32),
                    np.asarray(demands, dtype=np.float64), np.arange(n + 1, dtype=np.int64),
                    np.arange(n + 1, dtype=np.int64), np.zeros(n, np.int32), {})


def water_level(demands: np.ndarray, capacity: float) -> np.ndarray:
    """Fair shares on one link: S_c = min(D_c, l) with sum_c S_c = min(C, sum D)."""
    d = np.sort(np.asarray(demands, dtype=np.float64))
    if d.sum() <= capacity:
        return np.asarray(demands, dtype=np.float64).copy()
    rem = capacity
    n = d.shape[0]
    for i in range(n):
        share = rem / (n - i)
        if d[i] >= share:
            return np.minimum(np.asarray(demands, dtype=np.float64), share)
        rem -= d[i]
    raise AssertionError("unreachable")
