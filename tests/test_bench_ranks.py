"""Multi-rank aggregation of bench.py on CPU: two gloo ranks, each a replica with its own
step time; the job's rate is world_size iterations per step in the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cpu")
        bench.fence(dev)
        ms_local = 2.0 + 3.0 * rank             # rank 1 is the slow replica
        rate, ms = bench.job_rate(ms_local, world, dev)
        mx = bench.max_over_ranks(10.0 - rank, dev)
        bench.fence(dev)
        q.put((rank, rate, ms, mx, bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_rank_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms, mx, env in res:
        assert ms == 5.0                         # the slowest rank's step time on every rank
        assert rate == pytest.approx(world / 5e-3)
        assert mx == 10.0
        assert env == (rank, world, rank)


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms = bench.job_rate(4.0, 1, torch.device("cpu"))
    assert ms == 4.0 and rate == pytest.approx(250.0)
