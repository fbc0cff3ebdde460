"""The replica (N > 1) path of bench.py on CPU: two gloo ranks reduce their
timings to the slowest rank's, and the whole-job value counts every rank's
work over that time.  The GPU runs use the same functions over NCCL."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (1 + r) seconds on the device and (2 + r) end to end
    t_dev, t_e2e = bench.max_over_ranks([1.0 + rank, 2.0 + rank], world, None)
    dist.barrier()
    out.put((rank, t_dev, t_e2e, bench.replica_value(world, 100.0, t_dev)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_dev, t_e2e, value in res:
        assert t_dev == 2.0 and t_e2e == 3.0
        assert value == pytest.approx(2 * 100.0 / 2.0)


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.replica_value(1, 10.0, 2.0) == 5.0
