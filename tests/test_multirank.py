"""The multi-GPU path of bench.py runs one independent replica per rank and
reports all ranks' particle-steps over the slowest rank's time.  Here its
host-side logic runs as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_setup()
    # rank r "timed" 100 + 50 r ms for 1000 + r particles over 10 steps
    ms_max, value = bench.aggregate_ranks(100.0 + 50.0 * rank, 1000 + rank, 10, world)
    q.put((rank, w, r, lr, ms_max, value, bench.replica_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, lr, ms_max, value, seed in res:
        assert (w, r, lr) == (2, rank, rank)
        assert ms_max == 150.0                          # the slowest rank
        assert value == pytest.approx((1000 + 1001) * 10 / 0.150)
    assert res[0][6] != res[1][6]                       # independent replicas


def test_single_rank_aggregation():
    import bench
    ms_max, value = bench.aggregate_ranks(200.0, 5000, 20, 1)
    assert ms_max == 200.0 and value == pytest.approx(5000 * 20 / 0.2)
