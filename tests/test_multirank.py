"""The N > 1 host path of bench.py with two gloo ranks on CPU: each rank plans
its own seeded placement, the time is the slowest rank's, and the reported
rate counts the work of all ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w) == (rank, world)

        class A:
            grid = "40,36,32"
            fdtd_steps = 20
        case = bench.make_case(A, r)
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist)
        rate = bench.whole_job_rate(w, 3, case.voxels * 2 * case.n_steps, ms)
        out[rank] = (int(case.index.sum()), ms, rate, case.voxels)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_bookkeeping():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    (s0, ms0, rate0, vox), (s1, ms1, rate1, _) = out[0], out[1]
    assert s0 != s1                              # each rank its own seeded phantom
    assert ms0 == ms1 == 150.0                   # the slowest rank's time on every rank
    expected = world * 3 * vox * 2 * 20 / 0.150 / 1e9
    assert rate0 == rate1 == pytest.approx(expected, rel=1e-12)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.whole_job_rate(1, 2, 1e9, 1000.0) == pytest.approx(2.0)
