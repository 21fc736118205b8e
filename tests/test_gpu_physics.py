"""GPU parity of the Sigma-code options (half Coulomb-hole factor, screened-exchange
cutoff for negative frequencies) against the oracle, through the C ABI: FP64, FP32-bulk,
batched and the adjoint."""

import numpy as np
import pytest

import oracle
from paper_2008_11326_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def gpp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11326_gb300 import gpp as g
    return g


def rel_err(got, ref):
    got = np.concatenate([np.ravel(g) for g in got])
    ref = np.concatenate([np.ravel(r) for r in ref])
    nz = ref != 0
    assert np.all(got[~nz] == 0)
    return float(np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz]), initial=0.0))


def negative_frequency_problem(seed=91, B=10, G=600, P=7, W=3):
    """Frequencies of both signs and Re w spread over both signs, so that the cutoff
    drops some terms on branch 1 and on branch 2 and keeps others."""
    prob = inputs.make_problem(B, 2, G, P, W, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    wt = prob.wtilde_array.copy()
    wt.real *= rng.choice([-1.0, 1.0], size=wt.shape)
    wx = rng.uniform(-3.0, 3.0, size=(B, W))
    return prob.replace(wtilde_array=wt, wx_array=wx)


def run(gpp, prob, **opts):
    import torch
    dp = gpp.DeviceProblem.from_host(prob, device="cuda",
                                     c64=opts.get("precision") == "fp32_bulk")
    ach, asx = gpp.sigma(dp, **opts)
    torch.cuda.synchronize()
    return ach.cpu().numpy(), asx.cpu().numpy()


@pytest.mark.parametrize("ch_half,sexcut", [(True, 0.0), (False, 4.0), (True, 1.5), (False, 0.7)])
def test_fp64_matches_oracle(gpp, ch_half, sexcut):
    prob = negative_frequency_problem()
    ref = oracle.sigma(prob, ch_half=ch_half, sexcut=sexcut)
    if sexcut:  # the option changes the answer on this problem
        plain = oracle.sigma(prob, ch_half=ch_half)
        assert rel_err(plain, ref) > 1e-6
    assert rel_err(run(gpp, prob, ch_half=ch_half, sexcut=sexcut), ref) <= RTOL


def test_fp32_bulk_matches_oracle(gpp):
    prob = negative_frequency_problem(seed=92)
    ref = oracle.sigma(prob, ch_half=True, sexcut=2.0)
    got = run(gpp, prob, precision="fp32_bulk", ch_half=True, sexcut=2.0)
    assert rel_err(got, ref) <= 1e-6


def test_half_factor_is_exact_and_fast_path_unaffected(gpp):
    prob = inputs.make_problem(12, 2, 900, 9, 3, seed=93)   # all x >= 0: the fast path
    a0, s0 = run(gpp, prob)
    a1, s1 = run(gpp, prob, ch_half=True, sexcut=4.0)
    assert np.array_equal(a1, 0.5 * a0) and np.array_equal(s1, s0)


def test_batched_matches_oracle(gpp):
    import torch
    probs = [negative_frequency_problem(seed=s, B=b, G=g, P=p)
             for s, b, g, p in ((94, 5, 300, 4), (95, 9, 700, 6), (96, 3, 128, 3))]
    dps = [gpp.DeviceProblem.from_host(p, device="cuda") for p in probs]
    plan = gpp.BatchedPlan(dps, ch_half=True, sexcut=1.5)
    outs = plan.run()
    torch.cuda.synchronize()
    for (a, s), p in zip(outs, probs):
        ref = oracle.sigma(p, ch_half=True, sexcut=1.5)
        assert rel_err((a.cpu().numpy(), s.cpu().numpy()), ref) <= RTOL


def test_adjoint_matches_oracle(gpp):
    import torch
    prob = negative_frequency_problem(seed=97, B=6, G=300, P=5)
    ga, gs = inputs.cotangents(97, prob.nw)
    ref = oracle.sigma_adjoint(prob, ga, gs, ch_half=True, sexcut=1.5)
    dp = gpp.DeviceProblem.from_host(prob, device="cuda")
    got = gpp.sigma_backward(dp, torch.from_numpy(ga).cuda(), torch.from_numpy(gs).cuda(),
                             ch_half=True, sexcut=1.5)
    torch.cuda.synchronize()
    for k in ("wtilde", "I_eps", "aqsm", "aqsn"):
        g = got[k].cpu().numpy()
        scale = np.abs(ref[k]).max()
        assert np.max(np.abs(g - ref[k])) <= 1e-11 * scale, k


def test_autograd_function_carries_the_options(gpp):
    import torch
    prob = negative_frequency_problem(seed=98, B=4, G=200, P=3)
    dev = "cuda"
    t = {f: torch.from_numpy(np.ascontiguousarray(getattr(prob, f))).to(dev)
         for f in ("aqsmtemp", "aqsntemp", "I_eps_array", "wtilde_array", "vcoul",
                   "inv_igp_index", "indinv", "wx_array")}
    w = t["wtilde_array"].clone().requires_grad_(True)
    ach, asx = gpp.GppSigma.apply(t["aqsmtemp"], t["aqsntemp"], t["I_eps_array"], w, t["vcoul"],
                                  t["inv_igp_index"], t["indinv"], t["wx_array"], prob.nvband,
                                  "all", True, 1.5)
    ga, gs = inputs.cotangents(98, prob.nw)
    loss = (torch.real(torch.conj(torch.from_numpy(ga).to(dev)) * ach).sum()
            + torch.real(torch.conj(torch.from_numpy(gs).to(dev)) * asx).sum())
    loss.backward()
    ref = oracle.sigma_adjoint(prob, ga, gs, want=("wtilde",), ch_half=True, sexcut=1.5)
    g = w.grad.cpu().numpy()
    assert np.max(np.abs(g - ref["wtilde"])) <= 1e-11 * np.abs(ref["wtilde"]).max()
