"""Host logic of the multi-process path, on CPU with the gloo backend and
two ranks: independent instances are sharded without overlap, and the
whole-job rate divides all ranks' units by the slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = list(range(11))
    mine = bench.shard(items, rank, world)
    # rank r "processes" its share in (r + 1) seconds
    rate = bench.job_rate(float(len(mine)), float(rank + 1), world)
    slowest = bench.max_over_ranks(float(rank + 1), world)
    bench.barrier(world)
    q.put((rank, mine, rate, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (m, rate, slow)) for r, m, rate, slow in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(out[0][0] + out[1][0]) == list(range(11))
    assert not set(out[0][0]) & set(out[1][0])
    # 11 units in total over the slowest rank's 2 seconds, seen alike by both ranks
    assert out[0][1] == out[1][1] == pytest.approx(11 / 2.0)
    assert out[0][2] == out[1][2] == 2.0
