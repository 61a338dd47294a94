"""The N > 1 path of bench.py on CPU: two `gloo` ranks.

On N GPUs every rank runs its own replica of the workload (the solve does
not shard across GPUs here) and the job's time is the slowest rank's; the
reported value is the units all ranks processed over that time.  The
reference arm (the CPU oracle) runs on rank 0 alone.
"""
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


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = 100.0 * (rank + 1)            # rank 1 is the slower replica
        ms, value = bench.aggregate(torch, ms_local, 1000, world, "cpu")
        results[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_whole_job_time_is_the_slowest_rank_and_value_counts_all_ranks():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        results = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), results), nprocs=world,
                           start_method="spawn", join=True)
        out = dict(results)
    for rank in range(world):
        ms, value = out[rank]
        assert ms == 200.0
        assert value == pytest.approx(1000 * world / 0.2)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate(torch, 50.0, 10, 1, "cpu")
    assert ms == 50.0 and value == pytest.approx(200.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class Args:
        steps, warmup = 1, 0

    bench.run_reference(Args(), rank=1, world=2)
    assert capsys.readouterr().out == ""
