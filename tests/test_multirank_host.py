"""The replicated multi-rank path of bench.py (one solve per rank, no data-path
collective) on CPU: two gloo ranks, MAX of the timed region over ranks, SUM of
the units, and a barrier on both sides of the timed region."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, max_ms = bench.whole_job_rate(100.0 + 50.0 * rank, 1000.0 * (rank + 1))
    dist.barrier()
    out.put((rank, value, max_ms))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_as_the_driver_expects():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, max_ms in res:
        assert max_ms == 150.0                         # the slowest rank's time
        assert value == pytest.approx(3000.0 / 0.150)  # all ranks' units / that time


def test_single_process_returns_its_own_rate():
    sys.path.insert(0, ROOT)
    import bench
    value, max_ms = bench.whole_job_rate(200.0, 500.0)
    assert max_ms == 200.0 and value == pytest.approx(2500.0)
    assert bench.energy_reduction_launches(262144) == 2 and bench.energy_reduction_launches(1024) == 1
