"""The benchmark's multi-rank aggregation, run as two gloo ranks on CPU.

With N ranks (replicas, one per GPU) the benchmark takes every timing as the maximum over
the ranks and reports the whole job's rate: N x the per-rank work over that time. The
helpers that do this are the ones `bench.py` calls on the GPU path; here each rank passes a
different time and both must see the slower one.
"""

import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = 100.0 + 50.0 * rank          # rank 1 is the slower one
        m = bench.max_over_ranks(step_ms, dist)
        rate = bench.whole_job_tflops(4.37e12, m * 1e-3, world)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([m, rate]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_the_whole_job_work(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for m, rate in got:
        assert m == 150.0
        assert abs(rate - 2 * 4.37e12 / 0.150 / 1e12) < 1e-9


def test_single_process_is_the_identity():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_tflops(2e12, 1.0, 1) == 2.0
