"""GPU adjoint (gpp_sigma_backward / GppSigma) against the CPU reference adjoint and
against central finite differences of the oracle."""

import numpy as np
import pytest

import fd_restrict
import oracle
import oracle_pins as pins
from paper_2008_11326_gb300 import inputs

pytestmark = pytest.mark.gpu

KINDS = ("wtilde", "I_eps", "aqsm", "aqsn")


@pytest.fixture(scope="module")
def gpp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11326_gb300 import gpp as g
    return g


def gpu_grads(gpp, prob, ga, gs, occ="all"):
    import torch
    dp = gpp.DeviceProblem.from_host(prob, device="cuda")
    g = gpp.sigma_backward(dp, torch.from_numpy(ga).cuda(), torch.from_numpy(gs).cuda(),
                           occ_mode=occ)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in g.items()}


def max_rel(got, ref):
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / scale) if scale > 0 else float(np.abs(got).max())


@pytest.mark.parametrize("shape", [(4, 64, 8, 3), (5, 100, 13, 2), (3, 33, 9, 1),
                                   (9, 70, 17, 4)])
@pytest.mark.parametrize("occ", ["all", "occupied"])
def test_matches_cpu_adjoint_small(gpp, shape, occ):
    B, G, P, W = shape
    prob = inputs.make_problem(B, 2, G, P, W, seed=B * G + P)
    inv = prob.inv_igp_index.copy()
    inv[1] = prob.ncouls           # sentinel column
    inv[2] = inv[3]                # repeated global column
    prob = prob.replace(inv_igp_index=inv)
    ga, gs = inputs.cotangents(5, W)
    ref = oracle.sigma_adjoint(prob, ga, gs, occ_mode=0 if occ == "all" else 1)
    got = gpu_grads(gpp, prob, ga, gs, occ)
    for k in KINDS:
        assert max_rel(got[k], ref[k]) <= 1e-12, k


def test_general_path_inputs(gpp):
    prob = inputs.make_problem(6, 2, 96, 9, 3, seed=71)
    wt = prob.wtilde_array.copy()
    wt[0, :20] *= -1.0
    wx = np.linspace(-2.0, 3.5, 18).reshape(6, 3)
    prob = prob.replace(wtilde_array=wt, wx_array=wx)
    ga, gs = inputs.cotangents(6, 3)
    ref = oracle.sigma_adjoint(prob, ga, gs)
    got = gpu_grads(gpp, prob, ga, gs)
    for k in KINDS:
        assert max_rel(got[k], ref[k]) <= 1e-12, k


@pytest.mark.parametrize("wscale", [0.1, 0.05, 0.002])
def test_partial_fraction_bound(gpp, wscale):
    """As the forward's test of the same name: warps whose |w| reach down to max|wx| / 128
    take the fast path's partial fractions at their largest cancellation, smaller |w| the
    general form; every gradient within 1e-12 of the CPU adjoint."""
    from test_gpu_fwd import small_w_problem
    prob = small_w_problem(wscale)
    ga, gs = inputs.cotangents(8, 3)
    ref = oracle.sigma_adjoint(prob, ga, gs)
    got = gpu_grads(gpp, prob, ga, gs)
    for k in KINDS:
        assert max_rel(got[k], ref[k]) <= 1e-12, k


def test_closed_forms(gpp):
    for section, x in (("adjoint", 2.0), ("adjoint_branch2", 1.25)):
        g = pins.golden()[section]
        prob = pins.size1_problem(x, 1.0)
        for key, ga, gs in (("re_ach", 1.0, 0.0), ("im_asx", 0.0, 1j)):
            got = gpu_grads(gpp, prob, np.array([ga], np.complex128), np.array([gs], np.complex128))
            for name, want in g[key].items():
                assert abs(got[name][0, 0] - pins.cfrac(want)) <= 1e-13, (section, key, name)


def test_autograd_function(gpp):
    import torch
    prob = inputs.make_problem(5, 2, 80, 6, 3, seed=5)
    dev = "cuda"
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)  # noqa: E731
    leaves = [t(prob.aqsmtemp, torch.complex128).requires_grad_(),
              t(prob.aqsntemp, torch.complex128).requires_grad_(),
              t(prob.I_eps_array, torch.complex128).requires_grad_(),
              t(prob.wtilde_array, torch.complex128).requires_grad_()]
    ach, asx = gpp.GppSigma.apply(*leaves, t(prob.vcoul, torch.float64),
                                  t(prob.inv_igp_index, torch.int32),
                                  t(prob.indinv, torch.int32), t(prob.wx_array, torch.float64))
    a = torch.tensor([0.3, -1.2, 0.7], dtype=torch.float64, device=dev)
    b = torch.tensor([1.1, 0.4, -0.5], dtype=torch.float64, device=dev)
    L = (a * ach.real).sum() + (b * asx.imag).sum()
    L.backward()
    ref = oracle.sigma_adjoint(prob, a.cpu().numpy().astype(np.complex128),
                               1j * b.cpu().numpy())
    for leaf, k in zip(leaves, ("aqsm", "aqsn", "I_eps", "wtilde")):
        assert max_rel(leaf.grad.cpu().numpy(), ref[k]) <= 1e-12, k


def test_gradcheck_tiny(gpp):
    import torch
    prob = inputs.make_problem(2, 2, 6, 2, 2, seed=8)
    dev = "cuda"
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)  # noqa: E731
    fixed = (t(prob.vcoul, torch.float64), t(prob.inv_igp_index, torch.int32),
             t(prob.indinv, torch.int32), t(prob.wx_array, torch.float64))

    def f(aqsm, aqsn, eps, wt):
        return gpp.GppSigma.apply(aqsm, aqsn, eps, wt, *fixed)
    leaves = tuple(t(getattr(prob, n), torch.complex128).requires_grad_()
                   for n in ("aqsmtemp", "aqsntemp", "I_eps_array", "wtilde_array"))
    assert torch.autograd.gradcheck(f, leaves, eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.fixture(scope="module")
def adjoint_case():
    prob = inputs.config("adjoint")
    ga, gs = inputs.cotangents(3, prob.nw)
    return prob, ga, gs


@pytest.fixture(scope="module")
def adjoint_gpu(gpp, adjoint_case):
    prob, ga, gs = adjoint_case
    return gpu_grads(gpp, prob, ga, gs)


def test_adjoint_workload_vs_cpu_adjoint(adjoint_case, adjoint_gpu):
    """B=128, P=410, G=8192, nw=3; loss sum_iw a_iw Re ach + b_iw Im asx, a, b ~ N(0,1)."""
    prob, ga, gs = adjoint_case
    ref = oracle.sigma_adjoint(prob, ga, gs)
    for k in KINDS:
        assert max_rel(adjoint_gpu[k], ref[k]) <= 1e-12, k


def test_adjoint_workload_vs_finite_differences(orc, adjoint_case, adjoint_gpu):
    """64 random entries (16 per input); wtilde entries keep every term >= 10% away from the
    branch thresholds. Central differences with h = 1e-6 on the oracle."""
    prob, ga, gs = adjoint_case
    rng = np.random.Generator(np.random.PCG64(64))
    entries = pins.fd_entries(prob, 16, rng)
    assert len(entries) == 64
    worst = 0.0
    for kind, idx in entries:
        fd = fd_restrict.central_difference(orc, prob, ga, gs, kind, idx)
        adj = adjoint_gpu[kind][idx]
        err = abs(fd - adj) / max(abs(adj), 1e-2)
        worst = max(worst, err)
        assert err <= 1e-6, (kind, idx, fd, adj)
