"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own replica timing.
The job time is the slowest rank's (max over ranks on every rank), the value counts the
cell-stage updates of all ranks, and only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        local_s = 1.0 + 0.5 * r  # rank 1 is slower
        job_s = bench.reduce_max(local_s, w, device="cpu")
        out[r] = (w, r, local, job_s, bench.job_value(w, 100, 10, job_s))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        w, rr, local, job_s, value = out[r]
        assert (w, rr, local) == (world, r, r)
        assert job_s == 1.5
        assert value == world * 100 * 3 * 10 / 1.5


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=1, gpus=2)
    bench.run_reference(args, 2, 1)  # a non-zero rank returns at once, printing nothing
    assert capsys.readouterr().out == ""
