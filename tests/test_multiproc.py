"""The N>1 logic of bench.py on CPU ranks (gloo, world size 2): instance
sharding covers every lattice exactly once and the whole-job numbers take the
slowest rank's time and every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms, units = bench.reduce_over_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), ws)
    mine = bench.shard_indices(64, rank, ws)
    got = [None] * ws
    dist.all_gather_object(got, mine)
    out.put((rank, ms, units, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, shards in res:
        assert ms == 15.0  # slowest rank
        assert units == 300.0  # all ranks
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(64))
        assert abs(len(shards[0]) - len(shards[1])) <= 1


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.0, 7.0, 1) == (3.0, 7.0)
    assert bench.shard_indices(5, 0, 1) == [0, 1, 2, 3, 4]
