"""The multi-GPU path of bench.py on CPU: two gloo ranks.

With N > 1 every rank runs an independent replica (weak scaling) and the
job's throughput is the units of all ranks over the slowest rank's time;
only rank 0 prints.  These tests run that host logic with world_size 2 on
the gloo backend (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        # rank k: 100 (k + 1) ms for 1000 (k + 1) units per step, 10 steps
        value, max_ms, units = bench.job_throughput(100.0 * (rank + 1), 1000.0 * (rank + 1), 10, "cpu", world)
        out[rank] = (value, max_ms, units)
    finally:
        dist.destroy_process_group()


def test_job_throughput_is_all_units_over_the_slowest_rank():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        value, max_ms, units = out[rank]
        assert max_ms == pytest.approx(200.0)
        assert units == pytest.approx(3000.0)
        assert value == pytest.approx(3000.0 * 10 / 0.2)


def test_single_rank_needs_no_process_group():
    import bench

    value, max_ms, units = bench.job_throughput(50.0, 400.0, 5, "cpu", 1)
    assert (max_ms, units) == (50.0, 400.0)
    assert value == pytest.approx(400.0 * 5 / 0.05)


def test_reference_arm_is_rank0_only(capsys):
    import argparse

    import bench

    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1)  # returns at once, prints nothing
    assert capsys.readouterr().out == ""
