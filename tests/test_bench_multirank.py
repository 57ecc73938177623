"""The multi-rank arithmetic of bench.py on CPU: two gloo ranks, each with its own
step time; the job's time is the slowest rank's and the value counts every rank's
replica (weak scaling).  No GPU: the ranks exchange host numbers only."""
import os
import socket
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        total_ms = 100.0 + 50.0 * r  # rank 1 is slower
        job_ms = bench.max_over_ranks(total_ms)
        ms_per_step, value = bench.job_value(2899, w, job_ms, steps=10)
        with open(os.path.join(out_dir, f"rank{r}.txt"), "w") as f:
            f.write(f"{r} {w} {job_ms} {ms_per_step} {value}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_replica(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    rows = sorted(open(os.path.join(tmp_path, f"rank{r}.txt")).read().split() for r in range(2))
    for r, (rank, world, job_ms, ms_per_step, value) in enumerate(rows):
        assert int(rank) == r and int(world) == 2
        assert float(job_ms) == 150.0  # max over ranks
        assert float(ms_per_step) == pytest.approx(15.0)
        assert float(value) == pytest.approx(2 * 2899 / 15e-3)


def test_single_process_is_the_identity():
    assert bench.max_over_ranks(12.5) == 12.5
    ms, v = bench.job_value(100, 1, 50.0, 5)
    assert ms == 10.0 and v == pytest.approx(100 / 10e-3)
