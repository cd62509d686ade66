"""bench.py's multi-GPU mode is replicas only: each rank solves its own seeded
instances, the timed region is the slowest rank's, and the value counts every
rank's solves.  This checks that host logic with two gloo ranks on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [120.0, 250.0][rank]                 # rank 1 is the slow one
    mx = bench.replica_max_ms(elapsed, dist, "cpu")
    out.put((rank, mx, bench.replica_value(world, 3, mx),
             [bench.replica_seed(1002, s, rank) for s in range(3)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mx0, v0, s0), (r1, mx1, v1, s1) = res
    assert mx0 == mx1 == 250.0                     # max over ranks
    assert v0 == v1 == pytest.approx(2 * 3 / 0.25)  # 6 solves in 0.25 s
    assert not set(s0) & set(s1)                   # no instance solved twice
