"""Host logic of the batched tile autotuner: the proxy keeps every band and a fraction of
the igp columns (at least one)."""

import torch

from paper_2008_11326_gb300 import autotune, gpp, inputs


def test_proxy_keeps_bands_and_takes_a_column_fraction():
    for P, frac, want in ((1638, 1 / 32, 52), (102, 1 / 64, 2), (3, 1 / 64, 1), (8, 1.0, 8)):
        prob = inputs.make_problem(5, 2, max(P, 16), P, 3, seed=P)
        d = gpp.DeviceProblem.from_host(prob, device="cpu")
        q = autotune._proxy(d, frac)
        assert q.ngpown == want and q.number_bands == d.number_bands
        assert q.I_eps_array.shape[0] == want and q.inv_igp_index.shape[0] == want
        assert torch.equal(q.wtilde_array, d.wtilde_array[:want])
        assert q.aqsntemp is d.aqsntemp and q.wx_array is d.wx_array


def test_candidates_are_valid_launch_shapes():
    for bt, k in autotune.CANDIDATES:
        assert bt % 32 == 0 and 64 <= bt <= 256 and 1 <= k <= 8
