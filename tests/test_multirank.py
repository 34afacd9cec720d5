"""The benchmark's multi-rank path on CPU: world_size 2 over gloo.  Each
rank solves its own instance (no data exchange); the job figures are the max
of the ranks' timed regions and the sum of their units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate(1.5 + rank, 100 * (rank + 1))
    q.put((rank, t, u, bench.dist_info()))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, info in out:
        assert t == pytest.approx(2.5)
        assert u == pytest.approx(300.0)
        assert info[0] == rank and info[1] == 2


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(2.0, 7) == (2.0, 7.0)
