"""shard.sigma_columns on the GPU: with a one-rank NCCL group the column split and the
rank-ordered reduction wrapped around gpp_sigma give the unsharded result; with two gloo
ranks (two processes on the same GPU, each running gpp_sigma on its own column range, the
96-byte partials exchanged through host memory) the sum equals the oracle's."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2008_11326_gb300 import inputs

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_one_rank_nccl_column_sum_equals_gpp_sigma():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.distributed as dist
    from paper_2008_11326_gb300 import gpp, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("nccl", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        prob = inputs.make_problem(9, 2, 1500, 21, 3, seed=17)
        dp = gpp.DeviceProblem.from_host(prob, device="cuda")
        ach, asx = shard.sigma_columns(dp)
        ref_a, ref_s = gpp.sigma(dp)
        torch.cuda.synchronize()
        assert np.array_equal(ach.cpu().numpy(), ref_a.cpu().numpy())
        assert np.array_equal(asx.cpu().numpy(), ref_s.cpu().numpy())
    finally:
        dist.destroy_process_group()


def _gloo_rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    from paper_2008_11326_gb300 import gpp, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        prob = inputs.make_problem(9, 2, 1500, 21, 3, seed=17)
        dp = gpp.DeviceProblem.from_host(prob, device="cuda")
        for name, opts in (("fp64", {}), ("fp32_bulk", {"precision": "fp32_bulk"})):
            ach, asx = shard.sigma_columns(dp, **opts)
            torch.cuda.synchronize()
            np.save(os.path.join(out_dir, f"{name}_rank{rank}.npy"),
                    np.concatenate([ach.cpu().numpy(), asx.cpu().numpy()]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu_match_the_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    oracle.build()
    world = 2
    mp.spawn(_gloo_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    prob = inputs.make_problem(9, 2, 1500, 21, 3, seed=17)
    ref = np.concatenate(oracle.sigma(prob))
    for name, tol in (("fp64", 1e-12), ("fp32_bulk", 1e-6)):
        got = [np.load(tmp_path / f"{name}_rank{r}.npy") for r in range(world)]
        assert np.array_equal(got[0], got[1])      # every rank holds the same bits
        assert np.max(np.abs(got[0] - ref) / np.abs(ref)) <= tol, name
