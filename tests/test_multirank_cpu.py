"""The multi-GPU bench path is replicas only: one process per GPU, a barrier
and a max over ranks around the timed region, whole-job value = every rank's
bytes over the slowest rank's time, and the reference arm printed by rank 0
alone.  These run as two gloo ranks on the CPU (no GPU needed)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_local = 10.0 + 3.0 * rank          # rank 1 is the slow replica
        ms = bench.max_over_ranks(ms_local, world, dist, torch.device("cpu"))
        value = bench.job_value(world, 1 << 20, 5, ms)
        # only rank 1 saw a throttled clock: both ranks measure again
        again = bench.any_rank(rank == 1, world, dist, torch.device("cpu"))
        neither = bench.any_rank(False, world, dist, torch.device("cpu"))
        out[rank] = (ms, value, again, neither)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        ms, value, again, neither = res[r]
        assert ms == pytest.approx(13.0)                                   # max over ranks
        assert value == pytest.approx(world * (1 << 20) * 5 / 13e-3 / 1e9)  # all ranks' bytes / slowest time
        assert again is True and neither is False


def test_single_rank_is_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, None, None) == 7.5
    assert bench.job_value(1, 1000, 2, 1.0) == pytest.approx(1000 * 2 / 1e-3 / 1e9)


def test_reference_arm_prints_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(Args, rank=1, world=2)   # returns at once, no work
    assert buf.getvalue() == ""


def test_throttle_rule():
    sys.path.insert(0, ROOT)
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.throttled(ok)
    assert not bench.throttled({**ok, "sm_mhz": 1800.0, "reasons": ["sw_power_cap"]})   # power cap: kept
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.throttled({**ok, "reasons": [r]})
    assert bench.throttled({**ok, "sm_mhz": 1200.0})                  # far below max, no reason: a lock
    assert not bench.throttled({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})
    assert bench.any_rank(True, 1, None, None) and not bench.any_rank(False, 1, None, None)
