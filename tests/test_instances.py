"""The seeded instance generator: structure of the path sets it produces.

Paths must be valid, loopless walks from each demand's source to its
destination (flow conservation per demand: every unit sent on a path enters
at s and leaves at t), sorted by hop count, at most k per pair, and the
generator must be deterministic for a seed.
"""
from collections import deque

import numpy as np
import pytest

from paper_2605_01748_b300 import instances


def _check_paths(inst):
    src, dst = inst.edge_src, inst.edge_dst
    k = inst.meta["k"]
    for c in range(inst.n_demands):
        p0, p1 = inst.demand_path_off[c], inst.demand_path_off[c + 1]
        assert 1 <= p1 - p0 <= k
        prev_len = 0
        for r in range(p0, p1):
            es = inst.path_edges[inst.path_edge_off[r]:inst.path_edge_off[r + 1]]
            assert es.size >= 1
            assert src[es[0]] == inst.demand_src[c] and dst[es[-1]] == inst.demand_dst[c]
            assert (dst[es[:-1]] == src[es[1:]]).all(), "path is not a walk"
            nodes = np.concatenate([[src[es[0]]], dst[es]])
            assert np.unique(nodes).size == nodes.size, "path revisits a node"
            assert es.size >= prev_len, "paths not in non-decreasing hop order"
            prev_len = es.size


def _bfs_hops(inst, s):
    adj = [[] for _ in range(inst.n_nodes)]
    for a, b in zip(inst.edge_src, inst.edge_dst):
        adj[a].append(b)
    dist = [-1] * inst.n_nodes
    dist[s] = 0
    q = deque([s])
    while q:
        v = q.popleft()
        for w in adj[v]:
            if dist[w] < 0:
                dist[w] = dist[v] + 1
                q.append(w)
    return dist


def test_tiny_shape_and_paths(tiny):
    assert tiny.n_nodes == 12 and tiny.n_edges == 40 and tiny.n_demands == 132
    assert set(np.unique(tiny.capacity)) <= {100.0, 200.0, 400.0}
    assert np.isclose(tiny.demand.sum(), 0.5 * tiny.capacity.sum())
    _check_paths(tiny)
    # first path of every pair is a shortest path
    for s in range(tiny.n_nodes):
        dist = _bfs_hops(tiny, s)
        for c in np.where(tiny.demand_src == s)[0]:
            r = tiny.demand_path_off[c]
            assert tiny.path_edge_off[r + 1] - tiny.path_edge_off[r] == dist[tiny.demand_dst[c]]
    # both directions of a link share its capacity
    assert (tiny.capacity[0::2] == tiny.capacity[1::2]).all()


def test_deterministic(tiny):
    again = instances.make_tiny()
    assert again.digest() == tiny.digest()
    other = instances.make_tiny(seed=1)
    assert other.digest() != tiny.digest()


def test_medium_shape(medium):
    s = medium.summary()
    assert s["nodes"] == 200 and s["demands"] == 39800
    assert s["max_paths_per_demand"] == 8
    assert 550 <= s["links"] <= 650
    assert 5.0 <= s["mean_hops"] <= 7.0
    assert np.isclose(medium.demand.sum(), 0.5 * medium.capacity.sum())
    assert (medium.capacity >= 100).all() and (np.mod(medium.capacity, 100) == 0).all()
    sub = instances.subset(medium, np.arange(0, 39800, 97))
    _check_paths(sub)


def test_subset_roundtrip(tiny):
    sub = instances.subset(tiny, np.arange(tiny.n_demands))
    assert sub.digest() == tiny.digest()


def test_what_if_generator_shares_paths_within_a_scenario(tiny):
    W = instances.make_what_if(tiny, 3, 2, seed=1, min_fail=1, max_fail=2)
    assert len(W) == 6
    for s in range(3):
        a, b = W[2 * s], W[2 * s + 1]
        assert a.path_edges is b.path_edges and a.demand_path_off is b.demand_path_off
        failed = a.meta["failed_links"]
        dead = np.zeros(tiny.n_edges, bool)
        for l in failed:
            dead[2 * l] = dead[2 * l + 1] = True
        assert not dead[a.path_edges].any()
        assert (a.capacity[dead] == 0).all()
        assert (np.abs(a.demand / b.demand - 1) <= 0.5).all()


def test_drop_paths_keeps_the_chosen_paths(tiny):
    rng = np.random.default_rng(0)
    keep = rng.random(tiny.n_paths) < 0.5
    d = instances.drop_paths(tiny, keep)
    assert d.n_paths == int(keep.sum())
    kept = np.nonzero(keep)[0]
    for j, r in enumerate(kept):
        assert np.array_equal(d.path_edges[d.path_edge_off[j]:d.path_edge_off[j + 1]],
                              tiny.path_edges[tiny.path_edge_off[r]:tiny.path_edge_off[r + 1]])
    per = np.add.reduceat(keep.astype(int), tiny.demand_path_off[:-1])
    assert d.n_demands == int((per > 0).sum())
    assert np.array_equal(np.diff(d.demand_path_off), per[per > 0])
    assert np.array_equal(d.demand, tiny.demand[per > 0])
