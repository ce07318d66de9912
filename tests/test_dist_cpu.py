"""The multi-process path of the benchmark on CPU: two ranks over gloo
(127.0.0.1).  Ranks solve independent replicas, so the only collectives
are the barrier and the maximum of the timings; what-if instances are
dealt round robin with no exchange."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local, dist = bench.dist_setup(backend="gloo")
    assert (ws, r) == (world, rank)
    dist.barrier()
    m = bench.max_over_ranks([1.0 + rank, 10.0 * (world - rank), -rank], dist)
    out[rank] = (m, bench.shard(11, rank, world))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_and_sharding(world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        m, sh = res[r]
        assert m == [float(world), 10.0 * world, 0.0]
        assert sh == list(range(r, 11, world))
    assert sorted(i for r in range(world) for i in res[r][1]) == list(range(11))


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], None) == [3.0, 4.0]
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
