"""The N > 1 replica path of bench.py on CPU: two gloo ranks, barrier, max-over-ranks
timing and the whole-job throughput (every rank's units over the slowest rank's time)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t = 2.0 + rank                      # rank 1 is the slow one
    m = bench.barrier_max(world, t)
    rate = bench.replica_rate(world, 16, t)
    out.put((rank, m, rate))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_replicas_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, rate in res:
        assert m == pytest.approx(3.0)
        assert rate == pytest.approx(2 * 16 / 3.0)
