"""Column-sharded sums over two ranks with the gloo backend on CPU.

The per-rank partial sums come from the CPU oracle on each rank's column range (there is
no GPU here); the test covers the column split and the rank-ordered reduction that the GPU
path (shard.sigma_columns) uses unchanged.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2008_11326_gb300 import inputs, shard


def test_column_ranges_partition():
    for P in (0, 1, 7, 64, 1638):
        for world in (1, 2, 3, 8):
            ranges = [shard.column_range(P, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == P
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = inputs.make_problem(5, 2, 96, 13, 3, seed=71)
        lo, hi = shard.column_range(prob.ngpown, rank, world)
        a, s = oracle.sigma(prob.columns(slice(lo, hi)), nthreads=1)
        ach, asx = shard.reduce_outputs(torch.from_numpy(a), torch.from_numpy(s))
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.concatenate([ach.numpy(), asx.numpy()]))
    finally:
        dist.destroy_process_group()


def test_two_rank_column_split_equals_full_sum(tmp_path):
    import oracle
    oracle.build()
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    assert np.array_equal(got[0], got[1])           # every rank holds the same bits
    prob = inputs.make_problem(5, 2, 96, 13, 3, seed=71)
    ref = np.concatenate(oracle.sigma(prob))
    assert np.max(np.abs(got[0] - ref) / np.abs(ref)) <= 1e-13
