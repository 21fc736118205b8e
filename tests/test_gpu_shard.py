"""shard.sigma_columns on the GPU with a one-rank NCCL group: the column split and the
rank-ordered reduction wrapped around gpp_sigma give the unsharded result."""

import os
import socket

import numpy as np
import pytest

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
