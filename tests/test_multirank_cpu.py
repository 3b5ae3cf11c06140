"""The N > 1 host logic of bench.py on CPU: two gloo ranks (replicas), the
timing reduction takes the max over ranks, and the whole-job value counts the
units of all ranks over that time."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    t_max = bench.max_over_ranks(dist, local_ms, "cpu")
    out[rank] = (t_max, bench.whole_job_rate(world, 1.0e8, 10, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_value():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t_max, value = out[r]
        assert t_max == 150.0
        assert value == pytest.approx(2 * 1.0e8 * 10 / 0.150)


def test_single_process_identity():
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.whole_job_rate(1, 2.0, 4, 1000.0) == pytest.approx(8.0)
