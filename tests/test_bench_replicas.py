"""The multi-GPU path of bench.py is replicas only: every rank steps its own domain, the job time
is the slowest rank's, and the value is the whole job's throughput.  Checked here with two gloo
ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.max_over_ranks(times[rank], world, device="cpu")
    out[rank] = (t, bench.aggregate_mlups(1000, 10, world, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    times = [0.5, 2.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, v = out[r]
        assert t == 2.0
        assert v == pytest.approx(1000 * 10 * 2 / 2.0 / 1e6)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_mlups(1_179_648, 1000, 1, 0.1) == pytest.approx(11796.48)
