"""GPU parity of the FP64 forward sum against the CPU oracle, through the C-ABI.

Tolerance: every achtemp / asxtemp value within relative error 1e-12 of the oracle
(outputs that are zero by construction must be exactly zero).
"""

import numpy as np
import pytest

import oracle
import oracle_pins as pins
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


def run(gpp, prob, **opts):
    import torch
    dp = gpp.DeviceProblem.from_host(prob, device="cuda")
    ach, asx = gpp.sigma(dp, **opts)
    torch.cuda.synchronize()
    return ach.cpu().numpy(), asx.cpu().numpy()


def rel_err(got, ref):
    got = np.concatenate([np.ravel(g) for g in got])
    ref = np.concatenate([np.ravel(r) for r in ref])
    nz = ref != 0
    assert np.all(got[~nz] == 0), f"outputs that must be zero are {got[~nz]}"
    return float(np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz]), initial=0.0))


def check(gpp, prob, occ="all", **opts):
    got = run(gpp, prob, occ_mode=occ, **opts)
    ref = oracle.sigma(prob, occ_mode=0 if occ == "all" else 1)
    err = rel_err(got, ref)
    assert err <= RTOL, f"relative error {err:.3e}"
    return got, ref


def test_tiny_matches_oracle(gpp):
    check(gpp, inputs.config("tiny"))


@pytest.mark.parametrize("shape", [(5, 1000, 37, 3), (1, 1, 1, 1), (3, 129, 2, 8),
                                   (7, 300, 5, 5), (2, 64, 64, 2), (9, 257, 3, 4),
                                   (4, 4096, 1, 3)])
def test_ragged_sizes(gpp, shape):
    B, G, P, W = shape
    check(gpp, inputs.make_problem(B, 2, G, P, W, seed=B * 1000 + G))


def test_closed_forms(gpp):
    for case in pins.golden()["forward"]:
        from fractions import Fraction
        prob = pins.size1_problem(float(Fraction(case["x"])), pins.cfrac(case["w"]),
                                  inv=tuple(case.get("inv_igp_index", [0])),
                                  nvband=case.get("nvband", 1))
        occ = "occupied" if case.get("occ_mode", 0) == 1 else "all"
        ach, asx = run(gpp, prob, occ_mode=occ)
        want = np.array([pins.cfrac(case["ach"]), pins.cfrac(case["asx"])])
        got = np.array([ach[0], asx[0]])
        assert np.all(np.abs(got - want) <= 1e-13 + 1e-14 * np.abs(want)), (case["name"], got, want)


def test_index_case(gpp):
    g = pins.golden()["index_case"]
    ach, asx = run(gpp, pins.index_problem())
    want_a = np.array([pins.cfrac(v) for v in g["ach"]])
    want_s = np.array([pins.cfrac(v) for v in g["asx"]])
    assert np.allclose(ach, want_a, rtol=1e-14, atol=1e-13)
    assert np.allclose(asx, want_s, rtol=1e-14, atol=1e-13)


def test_general_path_branches(gpp):
    """Inputs outside the fast path: negative frequencies, Re w < 0, |w| large enough for
    LIMITONE to matter, |w| tiny enough for TOL_ZERO, frequencies next to w."""
    prob = inputs.make_problem(6, 2, 200, 6, 4, seed=77)
    wt = prob.wtilde_array.copy()
    wt[0, :50] *= -1.0                       # Re w < 0
    wt[1, :40] = 400.0 + 0.01j               # |delw| >= 500 possible -> LIMITONE
    wt[2, :30] = 1e-7 + 1e-8j                # |delw|^2 <= TOL_ZERO -> branch 3
    wx = np.linspace(-2.5, 3.5, 24).reshape(6, 4)   # negative x and x near Re w
    wx[5, :] = [400.3, 400.6, 399.7, 401.0]
    prob = prob.replace(wtilde_array=wt, wx_array=wx)
    branches = {oracle.branch(wt[p, ig], x) for p in range(3) for ig in range(0, 60, 7)
                for x in wx.ravel()}
    assert branches == {1, 2, 3}
    check(gpp, prob)


def test_near_threshold_fast_path(gpp):
    """Fast path with many terms next to |wdiff| = 1/2 (frequencies spread over Re w)."""
    prob = inputs.make_problem(8, 2, 512, 8, 3, seed=5)
    wx = np.linspace(0.0, 3.5, 24).reshape(8, 3)
    check(gpp, prob.replace(wx_array=wx))


def small_w_problem(wscale, seed=41):
    """Half of every column's G-vectors with |w| = wscale (Re w > 0, small phase), the rest
    as drawn; the largest frequency is 12."""
    prob = inputs.make_problem(24, 2, 512, 6, 3, seed=seed)
    wt = prob.wtilde_array.copy()
    ph = np.clip(np.angle(wt[:, :256]), -0.2, 0.2)
    wt[:, :256] = wscale * np.exp(1j * ph)
    wx = prob.wx_array.copy()
    wx[0, 2] = 12.0
    return prob.replace(wtilde_array=wt, wx_array=wx)


@pytest.mark.parametrize("wscale", [0.1, 0.05, 0.002])
def test_partial_fraction_bound(gpp, wscale):
    """The fast path's partial fractions lose bits where x >> |w|, so a warp takes them only
    if every |w| >= max|wx| / 128 (here 12 / 128 = 0.094): |w| = 0.1 puts warps on them at
    their largest cancellation (x / |w| up to 120), |w| = 0.05 and 0.002 send those warps to
    the general form (at 0.002 the partial fractions would lose ~13 bits, more than the
    1e-12 bar allows); the other warps are ordinary. All within 1e-12 of the oracle."""
    check(gpp, small_w_problem(wscale))


def test_occupied_mode(gpp):
    prob = inputs.make_problem(6, 2, 300, 7, 3, seed=9)
    check(gpp, prob, occ="occupied")
    check(gpp, prob.replace(nvband=0), occ="occupied")
    check(gpp, prob.replace(nvband=10), occ="occupied")


def test_sentinel_and_out_of_range_columns(gpp):
    from paper_2008_11326_gb300 import _native
    prob = inputs.make_problem(4, 2, 128, 6, 3, seed=12)
    inv = prob.inv_igp_index.copy()
    inv[1] = prob.ncouls                     # the sentinel
    sentinel = prob.replace(inv_igp_index=inv)
    check(gpp, sentinel, debug_checks=True)   # the sentinel is legitimate
    inv2 = inv.copy()
    inv2[3] = prob.ncouls + 5                # outside indinv: contributes nothing
    inv2[4] = -2
    bad = prob.replace(inv_igp_index=inv2)
    check(gpp, bad)
    with pytest.raises(_native.GppError, match="BAD_INDEX"):
        run(gpp, bad, debug_checks=True)


def test_deterministic_and_launch_shapes(gpp):
    prob = inputs.make_problem(16, 2, 2048, 40, 3, seed=31)
    a = run(gpp, prob)
    b = run(gpp, prob)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ref = oracle.sigma(prob)
    for bt in (64, 128, 256):
        for bps in (0, 1, 3):
            got = run(gpp, prob, block_threads=bt, blocks_per_sm=bps)
            assert rel_err(got, ref) <= RTOL, (bt, bps)
    for k in (1, 2, 3, 8):
        got = run(gpp, prob, ig_per_thread=k)
        assert rel_err(got, ref) <= RTOL, k


def test_empty_problems(gpp):
    for B, G, P in [(0, 16, 2), (3, 16, 0), (3, 0, 0)]:
        prob = inputs.make_problem(B, 2, G, P, 3, seed=1)
        ach, asx = run(gpp, prob)
        assert np.all(ach == 0) and np.all(asx == 0)


def test_column_and_band_splits_add_up(gpp):
    prob = inputs.make_problem(12, 2, 1500, 30, 3, seed=41)
    full = run(gpp, prob)
    c1 = run(gpp, prob.columns(slice(0, 13)))
    c2 = run(gpp, prob.columns(slice(13, None)))
    b1 = run(gpp, prob.bands(slice(0, 5)))
    b2 = run(gpp, prob.bands(slice(5, None)))
    for x, y in ((c1, c2), (b1, b2)):
        assert rel_err((x[0] + y[0], x[1] + y[1]), full) <= 1e-13


@pytest.mark.parametrize("pin", [True, False])
def test_host_entry_point_matches_device(gpp, pin):
    """Page-locked host arrays (aqsmtemp's gathered columns read in place by the gather
    kernel) and pageable ones (every input copied) give gpp_sigma's result bit for bit."""
    import torch
    prob = inputs.make_problem(6, 2, 700, 9, 3, seed=3)
    dev = run(gpp, prob)
    hp = gpp.DeviceProblem.from_host(prob, device="cpu", pin=pin)
    assert hp.aqsmtemp.is_pinned() == pin
    ws = torch.empty(gpp.host_workspace_size(hp), dtype=torch.uint8, device="cuda")
    ach, asx = gpp.sigma_host(hp, workspace=ws)
    assert np.array_equal(ach.numpy(), dev[0]) and np.array_equal(asx.numpy(), dev[1])


@pytest.mark.parametrize("shape", [(60, 9001, 1100), (24, 32768, 1100)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_host_entry_point_pipelined_chunks(gpp, precision, shape):
    """Instances large enough for the host entry to overlap its copies with the sum in
    G-vector chunks of doubling size on two streams ((2P + B) G 16 B = 330 MB: 2 chunks;
    1.2 GB: 8 chunks, the first of one G-vector tile): the result equals the device entry
    point's bit for bit (every tile keeps its partial slot and one reduction sums them in
    order), also with odd launch shapes and a ragged G."""
    import torch
    B, G, P = shape
    prob = inputs.make_problem(B, 2, G, P, 3, seed=8)
    dev = gpp.DeviceProblem.from_host(prob, device="cuda", c64=precision == "fp32_bulk")
    hp = gpp.DeviceProblem.from_host(prob, device="cpu", pin=True,
                                     c64=precision == "fp32_bulk")
    for opts in ({}, {"block_threads": 96, "ig_per_thread": 3}):
        a, s = gpp.sigma(dev, precision=precision, **opts)
        ws = torch.empty(gpp.host_workspace_size(hp, precision=precision, **opts),
                         dtype=torch.uint8, device="cuda")
        ha, hs = gpp.sigma_host(hp, workspace=ws, precision=precision, **opts)
        assert np.array_equal(ha.numpy(), a.cpu().numpy()), opts
        assert np.array_equal(hs.numpy(), s.cpu().numpy()), opts


def test_reciprocal_accuracy(gpp):
    import torch
    g = torch.Generator().manual_seed(0)
    x = torch.exp(torch.empty(1 << 20, dtype=torch.float64).uniform_(-30, 30, generator=g))
    x = x.cuda()
    got = gpp.rcp(x)
    ref = 1.0 / x
    rel = ((got - ref).abs() / ref.abs()).max().item()
    assert rel <= 4 * 2.0 ** -53, rel


@pytest.fixture(scope="module")
def benchmark_problem():
    return inputs.config("benchmark")


def test_benchmark_band_subsets_match_oracle(gpp, benchmark_problem):
    """The benchmark shape (B=512, P=1638, G=32768, nw=3): the oracle on 8-band subsets
    (the first 8 bands and 8 bands spread over the range) against the GPU on the same."""
    for sel in (slice(0, 8), np.arange(3, 512, 64)):
        sub = benchmark_problem.bands(sel)
        got = run(gpp, sub)
        ref = oracle.sigma(sub)
        assert rel_err(got, ref) <= RTOL


def test_benchmark_full_size_additivity(gpp, benchmark_problem):
    """The full benchmark launch (the configuration the benchmark times) equals the sum of
    64 launches over 8-band chunks, each of which is an oracle-checkable size."""
    full = run(gpp, benchmark_problem)
    acc_a = np.zeros(3, np.complex128)
    acc_s = np.zeros(3, np.complex128)
    for c in range(64):
        a, s = run(gpp, benchmark_problem.bands(slice(8 * c, 8 * c + 8)))
        acc_a += a
        acc_s += s
    assert rel_err((acc_a, acc_s), full) <= 1e-13


def test_side_stream_call_keeps_its_memory(gpp):
    """gpp.sigma on a stream other than the current one: the workspace and outputs it
    allocates are recorded on that stream, so memory freed when the call returns is not
    handed to the current stream (here a same-sized buffer filled right away) while the
    sum still runs."""
    import torch
    prob = inputs.make_problem(64, 2, 8192, 96, 3, seed=19)
    dp = gpp.DeviceProblem.from_host(prob, device="cuda")
    ref = np.concatenate([t.cpu().numpy() for t in gpp.sigma(dp)])
    need = gpp.workspace_size(dp)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        ach, asx = gpp.sigma(dp, stream=side)
        junk = torch.full((need,), 0x7f, dtype=torch.uint8, device="cuda")
        junk2 = torch.full((need,), 0x3c, dtype=torch.uint8, device="cuda")
        side.synchronize()
        got = np.concatenate([ach.cpu().numpy(), asx.cpu().numpy()])
        assert np.array_equal(got, ref)
        del junk, junk2
