"""The sliced device layout that te_create builds, checked on the host (no
GPU): tests/layout_check.cu is compiled against the library's layout builder
and run on seeded instances.  Every lane's ids must be exactly its path's
edges (any hop order) with the rest of the slot padded by the edge count E,
the per-lane hop counts must equal the path lengths, the block records must
match the slot and row offsets, and every demand must appear once with its
paths in order (path p of a demand on lane t*G + p%G, slot p/G)."""
import os
import subprocess

import numpy as np
import pytest

from paper_2605_01748_b300 import build, instances
from paper_2605_01748_b300.instances import Instance

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("layout") / "layout_check")
    cmd = [build._nvcc(), "-O2", "-std=c++17", "-I", build.INCLUDE, "-I", build.CSRC,
           os.path.join(HERE, "layout_check.cu"), os.path.join(build.CSRC, "te_layout.cu"), "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    return exe


def _run(checker, inst, tmp_path):
    d = str(tmp_path)
    inst.edge_src.astype(np.int32).tofile(os.path.join(d, "esrc.bin"))
    inst.edge_dst.astype(np.int32).tofile(os.path.join(d, "edst.bin"))
    inst.capacity.astype(np.float64).tofile(os.path.join(d, "cap.bin"))
    inst.demand.astype(np.float64).tofile(os.path.join(d, "dem.bin"))
    inst.demand_path_off.astype(np.int64).tofile(os.path.join(d, "dpo.bin"))
    inst.path_edge_off.astype(np.int64).tofile(os.path.join(d, "peo.bin"))
    inst.path_edges.astype(np.int32).tofile(os.path.join(d, "pe.bin"))
    res = subprocess.run([checker, d], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0 and res.stdout.startswith("OK"), res.stdout + res.stderr
    return res.stdout


def _ragged(seed, n_demands, max_paths, max_hops, n_edges=300):
    """Random demands with 1..max_paths paths of 1..max_hops edges each (the
    edges need not form walks: the layout does not look at the topology)."""
    rng = np.random.default_rng(seed)
    npaths = rng.integers(1, max_paths + 1, n_demands)
    dpo = np.concatenate([[0], np.cumsum(npaths)]).astype(np.int64)
    P = int(dpo[-1])
    plen = rng.integers(1, max_hops + 1, P)
    peo = np.concatenate([[0], np.cumsum(plen)]).astype(np.int64)
    pe = rng.integers(0, n_edges, int(peo[-1])).astype(np.int32)
    src = np.arange(n_edges, dtype=np.int32) % 7
    dst = (src + 1).astype(np.int32)
    return Instance(f"ragged-{seed}", 8, src, dst, rng.uniform(1.0, 5.0, n_edges), np.zeros(n_demands, np.int32),
                    np.ones(n_demands, np.int32), rng.uniform(0.5, 3.0, n_demands), dpo, peo, pe, {})


def test_layout_of_the_12_node_instance(checker, tmp_path):
    assert "G=1" in _run(checker, instances.make_tiny(), tmp_path)


def test_layout_of_the_200_node_instance(checker, tmp_path):
    assert "G=2" in _run(checker, instances.make_medium(), tmp_path)


@pytest.mark.parametrize("seed,max_paths,max_hops", [(1, 4, 12), (2, 16, 9), (3, 32, 40), (4, 7, 255)])
def test_layout_of_ragged_instances(checker, tmp_path, seed, max_paths, max_hops):
    _run(checker, _ragged(seed, 300, max_paths, max_hops), tmp_path)


@pytest.mark.parametrize("n_edges", [65534, 65535, 200000])
def test_layout_id_width_at_the_16_bit_limit(checker, tmp_path, n_edges):
    # 16-bit ids up to 65,534 edges (the sentinel E must fit), 32-bit above;
    # the checker asserts the width and reads every id back
    _run(checker, _ragged(5, 400, 8, 30, n_edges=n_edges), tmp_path)
