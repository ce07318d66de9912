"""Seeded synthetic TE instances (topology, capacities, demands, path sets).

This module is input generation only: it holds none of the TE method's
arithmetic and is the one piece of code that both the CPU oracle's tests and
the CUDA path consume.  The paper's inputs are a capacity edge list, a demand
matrix and a set of pre-computed paths per node pair (Section 3.1, Section 3.6
"Implementation"); its evaluation draws demands from a gravity model and uses
k-shortest paths (Section 4.2, "TE Inputs").  The public and production
topologies of the paper are not available here, so the instances below are
synthetic stand-ins with the shapes of those workloads:

* ``tiny``   -- 12-node ring plus 8 random chords (20 bidirectional links, 40
  directed edges), capacities uniform on {100, 200, 400}, all 132 ordered
  pairs with lognormal(0, 1) demands, k = 4.
* ``medium`` -- 200-node Waxman-type geometric WAN with ~600 links, lognormal
  capacities around 400 rounded to multiples of 100, gravity demands (Pareto
  node weights, shape 1.5) on all 39,800 ordered pairs, k = 8.
* ``large``  -- the same family with 1500 nodes, ~5,000 links (10,000 directed
  edges), ~2.25M demands, k = 16.

In every instance the total demand is half the total directed capacity.
Random numbers come from NumPy's PCG64 bit generator through ``random()``
only; normal and Pareto draws are formed here from those uniforms (Box-Muller,
inverse CDF) so the streams do not depend on NumPy's distribution code.
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import os
from typing import Optional

import numpy as np

from . import build as _build


@dataclasses.dataclass
class Instance:
    """A path-based TE instance in CSR form.

    Edges are directed; link ``i`` of the undirected topology owns edge ids
    ``2i`` (lower node id to higher) and ``2i + 1`` (the reverse), both with
    the same capacity.  Demand ``c`` owns paths
    ``demand_path_off[c] : demand_path_off[c+1]`` and path ``r`` traverses
    edges ``path_edges[path_edge_off[r] : path_edge_off[r+1]]`` in order.
    """

    name: str
    n_nodes: int
    edge_src: np.ndarray        # int32 [E]
    edge_dst: np.ndarray        # int32 [E]
    capacity: np.ndarray        # float64 [E]
    demand_src: np.ndarray      # int32 [K]
    demand_dst: np.ndarray      # int32 [K]
    demand: np.ndarray          # float64 [K]
    demand_path_off: np.ndarray  # int64 [K+1]
    path_edge_off: np.ndarray   # int64 [P+1]
    path_edges: np.ndarray      # int32 [nnz]
    meta: dict

    @property
    def n_edges(self) -> int:
        return int(self.capacity.shape[0])

    @property
    def n_demands(self) -> int:
        return int(self.demand.shape[0])

    @property
    def n_paths(self) -> int:
        return int(self.path_edge_off.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.path_edges.shape[0])

    def path_demand(self) -> np.ndarray:
        """Demand index of every path (int64 [P])."""
        counts = np.diff(self.demand_path_off)
        return np.repeat(np.arange(self.n_demands, dtype=np.int64), counts)

    def path_len(self) -> np.ndarray:
        return np.diff(self.path_edge_off)

    def digest(self) -> str:
        """SHA-256 over every array, so two consumers can check they saw the same input."""
        h = hashlib.sha256()
        for a in (self.edge_src, self.edge_dst, self.capacity, self.demand_src, self.demand_dst,
                  self.demand, self.demand_path_off, self.path_edge_off, self.path_edges):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()

    def summary(self) -> dict:
        pl = self.path_len()
        return {
            "name": self.name, "nodes": self.n_nodes, "edges": self.n_edges,
            "demands": self.n_demands, "paths": self.n_paths, "nnz": self.nnz,
            "mean_hops": float(pl.mean()) if pl.size else 0.0,
            "max_hops": int(pl.max()) if pl.size else 0,
            "max_paths_per_demand": int(np.diff(self.demand_path_off).max()) if self.n_demands else 0,
            **self.meta,
        }


# ---------------------------------------------------------------------------
# random draws (from PCG64 uniforms only)
# ---------------------------------------------------------------------------

def _uniform(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.random(n)


def _normal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform."""
    m = (n + 1) // 2
    u1 = 1.0 - rng.random(m)   # (0, 1]
    u2 = rng.random(m)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:n]


def _pareto(rng: np.random.Generator, n: int, xm: float, shape: float) -> np.ndarray:
    u = 1.0 - rng.random(n)    # (0, 1]
    return xm / u ** (1.0 / shape)


# ---------------------------------------------------------------------------
# topologies
# ---------------------------------------------------------------------------

def _ring_chords(rng: np.random.Generator, n: int, n_chords: int) -> list[tuple[int, int]]:
    links = [(min(i, (i + 1) % n), max(i, (i + 1) % n)) for i in range(n)]
    have = set(links)
    while len(links) < n + n_chords:
        u = int(rng.random() * n)
        v = int(rng.random() * n)
        if u == v:
            continue
        a, b = min(u, v), max(u, v)
        if (a, b) in have:
            continue
        have.add((a, b))
        links.append((a, b))
    return links


def _euclid_mst(pos: np.ndarray) -> list[tuple[int, int]]:
    """Prim's algorithm on the complete Euclidean graph (O(n^2))."""
    n = pos.shape[0]
    in_tree = np.zeros(n, dtype=bool)
    best = np.full(n, np.inf)
    parent = np.full(n, -1, dtype=np.int64)
    in_tree[0] = True
    d0 = np.linalg.norm(pos - pos[0], axis=1)
    best[:] = d0
    parent[:] = 0
    best[0] = np.inf
    links = []
    for _ in range(n - 1):
        cand = np.where(in_tree, np.inf, best)
        v = int(np.argmin(cand))
        in_tree[v] = True
        u = int(parent[v])
        links.append((min(u, v), max(u, v)))
        dv = np.linalg.norm(pos - pos[v], axis=1)
        upd = (~in_tree) & (dv < best)
        best[upd] = dv[upd]
        parent[upd] = v
        best[v] = np.inf
    return links


def _waxman(rng: np.random.Generator, n: int, n_links: int, locality: float) -> tuple[list[tuple[int, int]], np.ndarray]:
    """Waxman-type geometric graph: nodes uniform in the unit square, the
    Euclidean MST for connectivity, then extra links drawn independently with
    probability min(1, c * exp(-d / (locality * sqrt(2)))), c chosen so the
    expected link count is ``n_links``."""
    pos = rng.random((n, 2))
    mst = _euclid_mst(pos)
    have = set(mst)
    iu, ju = np.triu_indices(n, k=1)
    d = np.linalg.norm(pos[iu] - pos[ju], axis=1)
    w = np.exp(-d / (locality * np.sqrt(2.0)))
    mask = np.ones(iu.shape[0], dtype=bool)
    mst_arr = np.array(mst, dtype=np.int64)
    # linear index of (i, j), i < j, in the triu enumeration
    lin = mst_arr[:, 0] * n - mst_arr[:, 0] * (mst_arr[:, 0] + 1) // 2 + (mst_arr[:, 1] - mst_arr[:, 0] - 1)
    mask[lin] = False
    want = max(0, n_links - len(mst))
    wm = w[mask]
    lo, hi = 0.0, 1.0
    while np.minimum(1.0, hi * wm).sum() < want and hi < 1e30:
        hi *= 2.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if np.minimum(1.0, mid * wm).sum() < want:
            lo = mid
        else:
            hi = mid
    p = np.minimum(1.0, hi * w)
    u = rng.random(iu.shape[0])
    take = mask & (u < p)
    extra = list(zip(iu[take].tolist(), ju[take].tolist()))
    return mst + [(int(a), int(b)) for a, b in extra], pos


def _edges_from_links(links: list[tuple[int, int]]) -> tuple[np.ndarray, np.ndarray]:
    L = np.asarray(links, dtype=np.int32)
    src = np.empty(2 * len(links), dtype=np.int32)
    dst = np.empty(2 * len(links), dtype=np.int32)
    src[0::2], dst[0::2] = L[:, 0], L[:, 1]
    src[1::2], dst[1::2] = L[:, 1], L[:, 0]
    return src, dst


# ---------------------------------------------------------------------------
# k-shortest paths (native helper)
# ---------------------------------------------------------------------------

_gen_lib: Optional[ctypes.CDLL] = None


def _lib() -> ctypes.CDLL:
    global _gen_lib
    if _gen_lib is None:
        path = _build.build_gen()
        lib = ctypes.CDLL(path)
        lib.tegen_kpaths.restype = ctypes.c_int
        lib.tegen_kpaths.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
        lib.tegen_fetch.restype = ctypes.c_int
        lib.tegen_fetch.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 5
        lib.tegen_free.restype = None
        lib.tegen_free.argtypes = [ctypes.c_void_p]
        _gen_lib = lib
    return _gen_lib


def k_shortest_paths(n_nodes: int, edge_src: np.ndarray, edge_dst: np.ndarray, k: int,
                     max_hops: int = 64, threads: int = 0):
    """All-pairs k hop-shortest loopless paths (see csrc/gen/kpaths.cpp)."""
    order = np.lexsort((edge_dst, edge_src))
    adj_dst = np.ascontiguousarray(edge_dst[order], dtype=np.int32)
    adj_eid = np.ascontiguousarray(order, dtype=np.int32)
    adj_off = np.zeros(n_nodes + 1, dtype=np.int64)
    np.add.at(adj_off, edge_src.astype(np.int64) + 1, 1)
    adj_off = np.cumsum(adj_off)
    lib = _lib()
    handle = ctypes.c_void_p()
    counts = np.zeros(3, dtype=np.int64)
    rc = lib.tegen_kpaths(n_nodes, adj_off.ctypes.data, adj_dst.ctypes.data, adj_eid.ctypes.data,
                          k, max_hops, threads, ctypes.byref(handle), counts.ctypes.data)
    if rc != 0:
        raise RuntimeError("tegen_kpaths failed")
    try:
        K, P, nnz = (int(v) for v in counts)
        dsrc = np.empty(K, dtype=np.int32)
        ddst = np.empty(K, dtype=np.int32)
        dpo = np.empty(K + 1, dtype=np.int64)
        peo = np.empty(P + 1, dtype=np.int64)
        pe = np.empty(nnz, dtype=np.int32)
        rc = lib.tegen_fetch(handle, dsrc.ctypes.data, ddst.ctypes.data, dpo.ctypes.data,
                             peo.ctypes.data, pe.ctypes.data)
        if rc != 0:
            raise RuntimeError("tegen_fetch failed")
    finally:
        lib.tegen_free(handle)
    return dsrc, ddst, dpo, peo, pe


# ---------------------------------------------------------------------------
# instances
# ---------------------------------------------------------------------------

def _assemble(name: str, n: int, links, cap_link: np.ndarray, pair_demand, k: int,
              threads: int, meta: dict) -> Instance:
    esrc, edst = _edges_from_links(links)
    cap = np.repeat(np.asarray(cap_link, dtype=np.float64), 2)
    dsrc, ddst, dpo, peo, pe = k_shortest_paths(n, esrc, edst, k, threads=threads)
    D = pair_demand(dsrc, ddst)
    keep = D > 0
    if not keep.all():
        raise RuntimeError("generator produced a non-positive demand")
    D = D * (0.5 * cap.sum() / D.sum())
    return Instance(name=name, n_nodes=n, edge_src=esrc, edge_dst=edst, capacity=cap,
                    demand_src=dsrc, demand_dst=ddst, demand=D.astype(np.float64),
                    demand_path_off=dpo, path_edge_off=peo, path_edges=pe,
                    meta=dict(meta, k=k, links=len(links)))


def make_tiny(seed: int = 0, k: int = 4, threads: int = 0) -> Instance:
    """12-node ring plus 8 chords, capacities on {100, 200, 400}, all ordered
    pairs with lognormal(0, 1) demands scaled to half the total capacity."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 12
    links = _ring_chords(rng, n, 8)
    cap_link = np.array([100.0, 200.0, 400.0])[(rng.random(len(links)) * 3).astype(np.int64)]
    z = _normal(rng, n * n)
    lognorm = np.exp(z).reshape(n, n)

    def pair_demand(s, t):
        return lognorm[s, t]

    return _assemble("tiny", n, links, cap_link, pair_demand, k, threads,
                     {"seed": seed, "family": "ring+chords"})


def make_waxman(name: str, n: int, n_links: int, k: int, seed: int = 0, locality: float = 0.08,
                threads: int = 0) -> Instance:
    """Waxman-type WAN with lognormal capacities (median 400, sigma 0.5, rounded
    to multiples of 100, at least 100) and gravity demands w_s * w_t with
    Pareto(x_m = 1, shape 1.5) node weights."""
    rng = np.random.Generator(np.random.PCG64(seed))
    links, _ = _waxman(rng, n, n_links, locality)
    z = _normal(rng, len(links))
    raw = np.exp(np.log(400.0) + 0.5 * z)
    cap_link = np.maximum(100.0, 100.0 * np.round(raw / 100.0))
    wts = _pareto(rng, n, 1.0, 1.5)

    def pair_demand(s, t):
        return wts[s] * wts[t]

    return _assemble(name, n, links, cap_link, pair_demand, k, threads,
                     {"seed": seed, "family": "waxman", "locality": locality})


def make_medium(seed: int = 0, threads: int = 0) -> Instance:
    return make_waxman("medium", 200, 600, 8, seed=seed, locality=MEDIUM_LOCALITY, threads=threads)


def make_large(seed: int = 0, threads: int = 0) -> Instance:
    return make_waxman("large", 1500, 5000, 16, seed=seed, locality=LARGE_LOCALITY, threads=threads)


# locality of the Waxman family: tuned so the large instance's k = 16 paths
# average about six hops (~215M incidences) and the medium instance's k = 8
# paths about six hops (~1.9M incidences)
LARGE_LOCALITY = 0.05
MEDIUM_LOCALITY = 0.03


def make(name: str, seed: int = 0, threads: int = 0) -> Instance:
    if name == "tiny":
        return make_tiny(seed, threads=threads)
    if name == "medium":
        return make_medium(seed, threads=threads)
    if name == "large":
        return make_large(seed, threads=threads)
    if name == "wan3000":
        # beyond the shared-memory edge limit of the iteration kernel: 3000
        # nodes, 15,111 links (30,222 directed edges), all 8,997,000 ordered
        # pairs with their shortest path (k = 1)
        return make_waxman("wan3000", 3000, 15000, 1, seed=seed + 1, locality=LARGE_LOCALITY, threads=threads)
    raise ValueError(f"unknown instance {name!r}")


def subset(inst: Instance, demand_ids: np.ndarray, name: Optional[str] = None) -> Instance:
    """The sub-instance made of the given demands (all edges kept)."""
    demand_ids = np.asarray(demand_ids, dtype=np.int64)
    dpo = inst.demand_path_off
    npaths = dpo[demand_ids + 1] - dpo[demand_ids]
    new_dpo = np.concatenate([[0], np.cumsum(npaths)]).astype(np.int64)
    paths = np.concatenate([np.arange(dpo[c], dpo[c + 1]) for c in demand_ids]) if demand_ids.size else np.zeros(0, np.int64)
    plen = inst.path_edge_off[paths + 1] - inst.path_edge_off[paths]
    new_peo = np.concatenate([[0], np.cumsum(plen)]).astype(np.int64)
    pe = np.concatenate([inst.path_edges[inst.path_edge_off[r]:inst.path_edge_off[r + 1]] for r in paths]) \
        if paths.size else np.zeros(0, np.int32)
    return Instance(name=name or inst.name + "-subset", n_nodes=inst.n_nodes, edge_src=inst.edge_src,
                    edge_dst=inst.edge_dst, capacity=inst.capacity.copy(),
                    demand_src=inst.demand_src[demand_ids].copy(), demand_dst=inst.demand_dst[demand_ids].copy(),
                    demand=inst.demand[demand_ids].copy(), demand_path_off=new_dpo, path_edge_off=new_peo,
                    path_edges=pe.astype(np.int32), meta=dict(inst.meta))


def drop_paths(inst: Instance, keep_path: np.ndarray, name: Optional[str] = None) -> Instance:
    """The instance with only the paths where keep_path is true; demands left
    without a path are dropped (all edges kept)."""
    keep_path = np.asarray(keep_path, dtype=bool)
    dpo = inst.demand_path_off
    per_demand = np.add.reduceat(keep_path.astype(np.int64), dpo[:-1]) if inst.n_paths else np.zeros(0, np.int64)
    per_demand[np.diff(dpo) == 0] = 0
    dkeep = np.nonzero(per_demand > 0)[0]
    paths = np.nonzero(keep_path)[0]
    plen = inst.path_edge_off[paths + 1] - inst.path_edge_off[paths]
    new_peo = np.concatenate([[0], np.cumsum(plen)]).astype(np.int64)
    starts = inst.path_edge_off[paths]
    idx = np.repeat(starts - new_peo[:-1], plen) + np.arange(int(new_peo[-1]))
    pe = inst.path_edges[idx].astype(np.int32)
    new_dpo = np.concatenate([[0], np.cumsum(per_demand[dkeep])]).astype(np.int64)
    return Instance(name=name or inst.name + "-drop", n_nodes=inst.n_nodes, edge_src=inst.edge_src,
                    edge_dst=inst.edge_dst, capacity=inst.capacity.copy(),
                    demand_src=inst.demand_src[dkeep].copy(), demand_dst=inst.demand_dst[dkeep].copy(),
                    demand=inst.demand[dkeep].copy(), demand_path_off=new_dpo, path_edge_off=new_peo,
                    path_edges=pe, meta=dict(inst.meta))


def make_what_if(base: Instance, n_scenarios: int, n_matrices: int, seed: int = 0,
                 min_fail: int = 1, max_fail: int = 3, noise: float = 0.2) -> list:
    """What-if batch over one topology: n_scenarios failure scenarios, each
    removing min_fail..max_fail random links (both directions get capacity 0;
    the paths through them are dropped, and demands left without a path),
    times n_matrices demand matrices (the base demands times a lognormal
    factor clipped to 1 -/+ noise).  Instance s * n_matrices + m is scenario
    s with matrix m; its meta records the failed links."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_links = base.n_edges // 2
    factors = []
    for _ in range(n_matrices):
        z = _normal(rng, base.n_demands)
        factors.append(np.clip(np.exp(0.5 * noise * z), 1.0 - noise, 1.0 + noise))
    out = []
    for s in range(n_scenarios):
        nf = min_fail + int(rng.random() * (max_fail - min_fail + 1))
        failed = set()
        while len(failed) < nf:
            failed.add(int(rng.random() * n_links))
        dead = np.zeros(base.n_edges, dtype=bool)
        for l in failed:
            dead[2 * l] = dead[2 * l + 1] = True
        hit = np.add.reduceat(dead[base.path_edges].astype(np.int64), base.path_edge_off[:-1])
        keep = hit == 0
        keep[np.diff(base.path_edge_off) == 0] = False
        # the demand factors follow the demands that survive
        alive = np.add.reduceat(keep.astype(np.int64), base.demand_path_off[:-1]) > 0
        sc = drop_paths(base, keep, name=f"{base.name}-s{s}")
        sc.capacity[dead] = 0.0
        for m in range(n_matrices):
            inst = Instance(name=f"{base.name}-s{s}-m{m}", n_nodes=sc.n_nodes, edge_src=sc.edge_src,
                            edge_dst=sc.edge_dst, capacity=sc.capacity, demand_src=sc.demand_src,
                            demand_dst=sc.demand_dst, demand=sc.demand * factors[m][alive],
                            demand_path_off=sc.demand_path_off, path_edge_off=sc.path_edge_off,
                            path_edges=sc.path_edges,
                            meta=dict(base.meta, scenario=s, matrix=m, failed_links=sorted(failed)))
            out.append(inst)
    return out


def make_batch_base(seed: int = 0, threads: int = 0) -> Instance:
    """The 500-node WAN of the what-if batch: ~1,600 links, gravity demands on
    all 249,500 ordered pairs, k = 8."""
    return make_waxman("wan500", 500, 1600, 8, seed=seed, locality=MEDIUM_LOCALITY, threads=threads)
