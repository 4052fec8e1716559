"""The multi-process host logic of bench.py on CPU: two gloo ranks, each
timing its own replica, must agree on the slowest rank's time and report the
whole job's pixels over it (weak scaling: every rank decodes the full step).
The reference arm runs on rank 0 only; other ranks do no work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], ws)
        dist.barrier()
        out.put((rank, ms, bench.whole_job_mpix_s(1e6, 10, ws, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, times = 2, [12.5, 20.0]
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    mp.start_processes(_rank_main, args=(ws, _free_port(), times, out), nprocs=ws, join=True,
                       start_method="spawn")
    res = sorted(out.get() for _ in range(ws))
    for rank, ms, value in res:
        assert ms == max(times)
        # 2 ranks x 10 steps x 1 MPix in 20 ms = 1000 MPix/s
        assert value == pytest.approx(1000.0)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.0, 1) == 7.0
    assert bench.whole_job_mpix_s(2e6, 5, 1, 10.0) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank_zero_only():
    import bench
    assert bench.run_reference(None, 2, 1) is None
