"""Batched persistent launch (gpp_batched_plan_*): against per-instance gpp_sigma and the
oracle, graph replay, tile shapes, both precisions, and the autotuner."""

import numpy as np
import pytest

import oracle
from paper_2008_11326_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11326_gb300 import gpp as g
    return g


SHAPES = [(5, 300, 17, 3), (40, 1000, 37, 3), (3, 129, 2, 3), (70, 640, 32, 3),
          (9, 2048, 102, 3), (1, 64, 3, 3), (33, 777, 41, 3), (12, 256, 12, 3)]


@pytest.fixture(scope="module")
def batch():
    probs = []
    for i, (B, G, P, W) in enumerate(SHAPES):
        p = inputs.make_problem(B, 2, G, P, W, seed=2000 + i)
        if i == 1:  # a sentinel column
            inv = p.inv_igp_index.copy()
            inv[3] = p.ncouls
            p = p.replace(inv_igp_index=inv)
        probs.append(p)
    return probs


def device_batch(gpp, probs, c64=False):
    return [gpp.DeviceProblem.from_host(p, device="cuda", c64=c64) for p in probs]


def as_np(outs):
    return [np.concatenate([a.cpu().numpy(), s.cpu().numpy()]) for a, s in outs]


def max_rel(a, b):
    return max(float(np.max(np.abs(x - y) / np.abs(y))) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batched_matches_single_instance_calls(gpp, batch, precision, use_graph):
    import torch
    dps = device_batch(gpp, batch, c64=precision == "fp32_bulk")
    single = [gpp.sigma(d, precision=precision) for d in dps]
    plan = gpp.BatchedPlan(dps, use_graph=use_graph, precision=precision)
    outs = plan.run()
    torch.cuda.synchronize()
    assert max_rel(as_np(outs), as_np(single)) <= 1e-13
    first = as_np(outs)
    plan.run()
    torch.cuda.synchronize()
    for x, y in zip(as_np(plan.outputs), first):
        assert np.array_equal(x, y)  # replay is bit-for-bit identical
    plan.close()


def test_batched_fp64_matches_oracle(gpp, batch):
    import torch
    dps = device_batch(gpp, batch)
    plan = gpp.BatchedPlan(dps, precision="fp64")
    got = as_np(plan.run())
    torch.cuda.synchronize()
    ref = [np.concatenate(oracle.sigma(p)) for p in batch]
    assert max_rel(got, ref) <= 1e-12


@pytest.mark.parametrize("bt,k", [(64, 1), (128, 2), (256, 4), (96, 3)])
def test_tile_shapes(gpp, batch, bt, k):
    import torch
    dps = device_batch(gpp, batch)
    ref = [np.concatenate(oracle.sigma(p)) for p in batch]
    plan = gpp.BatchedPlan(dps, block_threads=bt, ig_per_thread=k)
    got = as_np(plan.run())
    torch.cuda.synchronize()
    assert max_rel(got, ref) <= 1e-12


def test_occupied_mode(gpp, batch):
    import torch
    dps = device_batch(gpp, batch)
    plan = gpp.BatchedPlan(dps, occ_mode="occupied")
    got = as_np(plan.run())
    torch.cuda.synchronize()
    ref = [np.concatenate(oracle.sigma(p, occ_mode=1)) for p in batch]
    assert max_rel(got, ref) <= 1e-12


def test_autotuner(gpp, batch, tmp_path, monkeypatch):
    from paper_2008_11326_gb300 import autotune
    monkeypatch.setenv("GPP_TUNE_CACHE", str(tmp_path / "tune.json"))
    dps = device_batch(gpp, batch)
    r = autotune.tune_batched(dps, proxy_fraction=0.25, reps=1)
    assert (r["block_threads"], r["ig_per_thread"]) in autotune.CANDIDATES and not r["cached"]
    assert autotune.tune_batched(dps, proxy_fraction=0.25, reps=1)["cached"]


def test_rejects_mixed_nw(gpp):
    from paper_2008_11326_gb300 import _native
    a = inputs.make_problem(3, 2, 64, 4, 3, seed=1)
    b = inputs.make_problem(3, 2, 64, 4, 2, seed=2)
    with pytest.raises(_native.GppError, match="nw"):
        gpp.BatchedPlan(device_batch(gpp, [a, b]))


def _host_problem(d, nb):
    """The first nb bands of a device instance, as host arrays for the oracle."""
    return inputs.GppProblem(
        number_bands=nb, nvband=d.nvband, ncouls=d.ncouls, ngpown=d.ngpown, nw=d.nw,
        aqsmtemp=d.aqsmtemp[:nb].cpu().numpy(), aqsntemp=d.aqsntemp[:nb].cpu().numpy(),
        I_eps_array=d.I_eps_array.cpu().numpy(), wtilde_array=d.wtilde_array.cpu().numpy(),
        vcoul=d.vcoul.cpu().numpy(), inv_igp_index=d.inv_igp_index.cpu().numpy(),
        indinv=d.indinv.cpu().numpy(), wx_array=d.wx_array[:nb].cpu().numpy())


def test_batched_workload_against_oracle(gpp):
    """The 64-instance batched workload (G log-uniform in [2048, 32768], P = G/20, B in
    64..512, drawn on the device), every instance cut to its first 8 bands so that the
    oracle takes seconds: one graph-replayed persistent launch over all 64, and four
    instances (smallest and largest G, two in between) against the oracle, FP64 and
    FP32-bulk."""
    import torch
    nb = 8
    full = [gpp.DeviceProblem(**inputs.make_device_arrays(**s, device="cuda"))
            for s in inputs.batched_shapes()]
    sub = [gpp.DeviceProblem(nb, d.nvband, d.ncouls, d.ngpown, d.nw, d.aqsmtemp[:nb],
                             d.aqsntemp[:nb], d.I_eps_array, d.wtilde_array, d.vcoul,
                             d.inv_igp_index, d.indinv, d.wx_array[:nb]) for d in full]
    order = sorted(range(len(sub)), key=lambda i: sub[i].ncouls)
    picks = [order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]]
    refs = {i: np.concatenate(oracle.sigma(_host_problem(full[i], nb))) for i in picks}
    for precision, tol in (("fp64", 1e-12), ("fp32_bulk", 1e-6)):
        plan = gpp.BatchedPlan(sub, use_graph=True, precision=precision)
        outs = as_np(plan.run())
        torch.cuda.synchronize()
        plan.close()
        for i in picks:
            err = float(np.max(np.abs(outs[i] - refs[i]) / np.abs(refs[i])))
            assert err <= tol, (precision, i, sub[i].ncouls, err)
    del full, sub
    torch.cuda.empty_cache()
