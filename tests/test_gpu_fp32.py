"""GPU parity of the FP32-bulk forward (GPP_FP32_BULK) against the FP64 oracle.

Target: relative error <= 1e-6 on each achtemp / asxtemp value.
"""

import numpy as np
import pytest

import oracle
from paper_2008_11326_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-6


@pytest.fixture(scope="module")
def gpp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11326_gb300 import gpp as g
    return g


def run(gpp, prob, precision="fp32_bulk", **opts):
    import torch
    dp = gpp.DeviceProblem.from_host(prob, device="cuda", c64=(precision == "fp32_bulk"))
    ach, asx = gpp.sigma(dp, precision=precision, **opts)
    torch.cuda.synchronize()
    return ach.cpu().numpy(), asx.cpu().numpy()


def rel_err(got, ref):
    got = np.concatenate([np.ravel(g) for g in got])
    ref = np.concatenate([np.ravel(r) for r in ref])
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def test_tiny(gpp):
    prob = inputs.config("tiny")
    assert rel_err(run(gpp, prob), oracle.sigma(prob)) <= RTOL


@pytest.mark.parametrize("shape", [(5, 1000, 37, 3), (3, 129, 2, 8), (40, 700, 9, 1),
                                   (70, 300, 4, 4)])
def test_ragged_and_chunk_tails(gpp, shape):
    B, G, P, W = shape
    prob = inputs.make_problem(B, 2, G, P, W, seed=B + G)
    assert rel_err(run(gpp, prob), oracle.sigma(prob)) <= RTOL


def test_decisions_next_to_the_branch_threshold(gpp):
    """Frequencies spread densely over the range of Re w put many terms within FP32
    rounding of |wdiff| = 1/2; a wrong branch decision would cost ~1e-4 here."""
    prob = inputs.make_problem(64, 2, 2048, 16, 3, seed=17)
    wx = np.linspace(0.0, 3.6, 192).reshape(64, 3)
    prob = prob.replace(wx_array=wx)
    assert rel_err(run(gpp, prob), oracle.sigma(prob)) <= RTOL


def test_next_to_the_wdiff_pole(gpp):
    """Real w with frequencies 1e-9 away from Re w: |wdiff|^2 is 0 in FP32 and 1e-18 in
    FP64. The branch-2 coefficient is taken in FP64 there; the result stays finite. (No
    frequency equals a w exactly: that is the pole itself, where the sum is undefined.)"""
    prob = inputs.make_problem(6, 2, 256, 4, 3, seed=23)
    wt = prob.wtilde_array.copy()
    vals = np.array([0.75, 1.25, 2.0, 2.5])
    wt[:, :64] = np.tile(vals, 16)[None, :] + 0j
    wx = np.array([[0.75 + 1e-9, 1.25 + 1e-9, 5.0], [2.0 + 1e-9, 2.5 - 1e-9, 0.3],
                   [1.0, 2.2, 3.0], [4.0, 5.0, 6.0], [0.75 + 2e-9, 7.0, 8.0],
                   [9.0, 2.5 + 3e-9, 1.25 - 1e-9]])
    prob = prob.replace(wtilde_array=wt, wx_array=wx)
    got = run(gpp, prob)
    assert all(np.all(np.isfinite(g)) for g in got)
    assert rel_err(got, oracle.sigma(prob)) <= RTOL


def test_band_frequencies_on_both_sides_of_the_warp_interval(gpp):
    """Re w in a narrow range, so a band can put one frequency below every Re w of a warp and
    another above (the per-band range test fails, each frequency is tested alone), next to
    bands entirely above or below, and bands straddling the interval."""
    prob = inputs.make_problem(12, 2, 700, 6, 3, seed=81)
    wt = prob.wtilde_array.copy()
    wt.real = 1.0 + 0.1 * (wt.real - 0.2) / 2.8
    wx = np.array([[0.1, 3.0, 0.2], [0.0, 0.3, 2.9], [2.0, 2.5, 4.0], [0.05, 0.1, 0.15],
                   [1.0, 1.05, 3.0], [0.4, 1.6, 0.45], [5.0, 0.0, 5.0], [1.2, 1.3, 1.4],
                   [0.2, 0.7, 2.4], [3.3, 0.33, 1.55], [0.0, 0.0, 0.0], [9.0, 8.0, 7.0]])
    prob = prob.replace(wtilde_array=wt, wx_array=wx)
    assert rel_err(run(gpp, prob), oracle.sigma(prob)) <= RTOL
    assert rel_err(run(gpp, prob, precision="fp64"), oracle.sigma(prob)) <= 1e-12


def test_frequencies_at_the_edges_of_the_warp_interval(gpp):
    """Every Re w = 1 and Im w = 0, so a warp's interval is [1/2 - 2^-20, 3/2 + 2^-20]
    (rounded outwards). Frequencies a few 1e-7 inside either end are on branch 2, just
    outside on branch 1: the per-lane path's bounds on x (formed from x_hi) must not call an
    inside frequency outside, which would put it on branch 1 (a ~1e-4 error). No frequency
    is 1 itself (the pole)."""
    prob = inputs.make_problem(8, 2, 512, 4, 3, seed=5)
    wt = np.full_like(prob.wtilde_array, 1.0 + 0.0j)
    e = 2.0 ** -20
    wx = np.array([[1.5 - 1e-7, 1.5 - 3e-7, 1.5 + e - 1e-7], [0.5 + 1e-7, 0.5 + 3e-7, 0.5 - e + 1e-7],
                   [1.5 + e + 1e-7, 0.5 - e - 1e-7, 1.1], [1.5 + 1e-6, 0.5 - 1e-6, 2.0],
                   [1.4999999, 1.5000001, 0.4999999], [0.5000001, 3.0, 0.0],
                   [1.5 + e, 0.5 - e, 1.25], [1.5, 0.5, 0.75]])
    prob = prob.replace(wtilde_array=wt, wx_array=wx)
    assert rel_err(run(gpp, prob), oracle.sigma(prob)) <= RTOL
    assert rel_err(run(gpp, prob, precision="fp64"), oracle.sigma(prob)) <= 1e-12


def test_general_inputs_take_the_fp64_path(gpp):
    prob = inputs.make_problem(6, 2, 200, 6, 4, seed=77)
    wx = np.linspace(-2.5, 3.5, 24).reshape(6, 4)     # negative x
    prob = prob.replace(wx_array=wx)
    assert rel_err(run(gpp, prob), oracle.sigma(prob)) <= 1e-12


def test_occupied_mode(gpp):
    prob = inputs.make_problem(40, 2, 600, 7, 3, seed=9)
    assert rel_err(run(gpp, prob, occ_mode="occupied"), oracle.sigma(prob, occ_mode=1)) <= RTOL


def test_occupied_split_inside_a_chunk_sorted(gpp):
    """Sorted passes (>= 128 bands) with the occupied bands ending inside a 16-band chunk
    (nvband = 21): the chunk's band sums run through both instantiations of the band body,
    and the Kahan compensation carried in the chunk sums crosses the split; ragged G."""
    prob = inputs.make_problem(131, 21, 1000, 8, 3, seed=131)
    for occ, mode in (("occupied", 1), ("all", 0)):
        got = run(gpp, prob, occ_mode=occ)
        assert rel_err(got, oracle.sigma(prob, occ_mode=mode)) <= RTOL, occ


def test_one_frequency_deep_tiles_sorted(gpp):
    """nw = 1, 160 threads x 8 G-vectors: the sort keys of a tile (1280 positions padded to
    2048 floats) outnumber the threads' shared-memory slots (160 x 12 floats), so the slot
    area is sized by the keys; the whole tile sorted (160 is not a power of two), ragged G."""
    prob = inputs.make_problem(128, 2, 1500, 5, 1, seed=12)
    got = run(gpp, prob, block_threads=160, ig_per_thread=8)
    assert rel_err(got, oracle.sigma(prob)) <= RTOL


def test_deterministic(gpp):
    prob = inputs.make_problem(33, 2, 1024, 20, 3, seed=4)
    a = run(gpp, prob)
    b = run(gpp, prob)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("nw", [1, 6, 7, 8])
def test_launch_shapes(gpp, nw):
    """Every CTA size and tile depth; at nw >= 7 and 256 threads the compensated pairs
    need more than 48 KB of shared memory per CTA."""
    prob = inputs.make_problem(37, 2, 900, 5, nw, seed=60 + nw)
    ref = oracle.sigma(prob)
    for bt in (64, 96, 128, 256):
        for k in (1, 4):
            assert rel_err(run(gpp, prob, block_threads=bt, ig_per_thread=k), ref) <= RTOL, (bt, k)


def test_sorted_passes_launch_shapes(gpp):
    """From 128 bands on the kernel sorts G-vectors by Re w before the band loop: within
    each pass of a tile when the block size is a power of two (128 x 3: the sort array is
    padded to 512 and its fourth segment is all padding), else over the whole tile (96 x 3:
    288 G-vectors padded to 512); a ragged G leaves inert positions in the last tile. Every
    shape sums the same FP32 terms in another order, so the shapes agree with each other
    more closely than with the oracle, and a G-vector skipped or taken twice would move an
    output by ~1e-3."""
    prob = inputs.make_problem(160, 2, 3001, 7, 3, seed=91)
    ref = oracle.sigma(prob)
    outs = []
    for bt, k in ((128, 4), (128, 3), (96, 3), (64, 1), (256, 2)):
        got = run(gpp, prob, block_threads=bt, ig_per_thread=k)
        assert rel_err(got, ref) <= RTOL, (bt, k)
        outs.append(np.concatenate(got))
    for o in outs[1:]:
        assert np.max(np.abs(o - outs[0]) / np.abs(outs[0])) <= 3e-7


def test_conversion_in_the_call_equals_a_kept_copy(gpp):
    """Without a caller's complex64 copy the call converts aqsntemp into its workspace; the
    result is the same, bit for bit, as with the copy made by gpp_convert_c64 and kept
    (tiny workload)."""
    import torch
    prob = inputs.config("tiny")
    dp = gpp.DeviceProblem.from_host(prob, device="cuda")
    a1, s1 = gpp.sigma(dp, precision="fp32_bulk")
    dp.make_c64()
    want = torch.from_numpy(prob.aqsntemp.astype(np.complex64)).cuda()
    assert torch.equal(dp.aqsntemp_c64, want)
    a2, s2 = gpp.sigma(dp, precision="fp32_bulk")
    torch.cuda.synchronize()
    assert torch.equal(a1, a2) and torch.equal(s1, s2)
    assert rel_err((a1.cpu().numpy(), s1.cpu().numpy()), oracle.sigma(prob)) <= RTOL


def test_benchmark_shape_band_subset(gpp):
    prob = inputs.config("mixed").bands(slice(0, 8))
    assert rel_err(run(gpp, prob), oracle.sigma(prob)) <= RTOL


def test_benchmark_shape_full_vs_fp64(gpp):
    """Full mixed-precision workload (B=512, P=1638, G=32768, nw=3) against the FP64 GPU
    path, which itself matches the oracle to 1e-12."""
    prob = inputs.config("mixed")
    f32 = run(gpp, prob)
    f64 = run(gpp, prob, precision="fp64")
    assert rel_err(f32, f64) <= RTOL
