"""The kernels' fast-path algebra, restated with numpy, against the oracle on the CPU.

On the fast path (x >= 0, Re w >= 0, 1e-12 < |w|^2 < 62499) branch 1 is |x - w|^2 > 1/4 and
branch 3 never occurs (test_fast_path_branch.py). The FP64 forward and adjoint kernels
then take the asxtemp terms in partial fractions instead of the written formulas: with
K = M I w, A = x - w and S = x + w,

  branch 1:  sch term K/A,  ssx term K w/(A S) = (K/A - K/S)/2   (S - A = 2 w)
  branch 2:  ssx term -(I delw)/(4 delw + 2) M = -K/(2 S)        (4 delw + 2 = 2 S/A)

so asxtemp = (achtemp over the occupied bands - sum K/S)/2, and for the adjoint, with
u = 1/A and v = 1/S, w u v = (u - v)/2 and 2 x^2 w (u v)^2 = x (u^2 - v^2)/2. This file
evaluates those forms directly (vectorised, FP64) and requires the oracle's results, which
follow the written formulas, to 1e-12; a wrong sign or factor in either identity fails it.
"""

import numpy as np
import pytest

import oracle
from paper_2008_11326_gb300 import inputs


def terms(prob):
    """Per (b, p, ig, iw): K, A, S, x and the branch-1 mask, and M, w, I, am, the
    gathered columns' validity (columns outside [0, G) contribute nothing)."""
    G = prob.ncouls
    k = prob.inv_igp_index.astype(np.int64)
    ok = (k >= 0) & (k <= G)
    g = np.where(ok, prob.indinv[np.clip(k, 0, G)], -1).astype(np.int64)
    valid = (g >= 0) & (g < G)
    gs = np.where(valid, g, 0)
    am = np.conj(prob.aqsmtemp[:, gs]) * prob.vcoul[gs][None, :] * valid[None, :]   # [B][P]
    M = am[:, :, None] * prob.aqsntemp[:, None, :]                                    # [B][P][G]
    w = prob.wtilde_array[None, :, :, None]
    I = prob.I_eps_array[None, :, :, None]
    x = prob.wx_array[:, None, None, :]
    K = M[..., None] * I * w
    A, S = x - w, x + w
    b1 = np.abs(A) ** 2 > 0.25
    return K, A, S, x, b1, M, w, I, am, gs, valid


def occ_mask(prob, occ_mode):
    B = prob.number_bands
    occ = np.ones(B) if occ_mode == 0 else (np.arange(B) < prob.nvband).astype(float)
    return occ[:, None, None, None]


def forward_partial_fractions(prob, occ_mode=0):
    K, A, S, x, b1, *_ = terms(prob)
    occ = occ_mask(prob, occ_mode)
    ach_terms = np.where(b1, K / A, 0.0)
    ach = ach_terms.sum(axis=(0, 1, 2))
    asx = 0.5 * (occ * (ach_terms - K / S)).sum(axis=(0, 1, 2))
    return ach, asx


def adjoint_partial_fractions(prob, g_ach, g_asx, occ_mode=0):
    K, A, S, x, b1, M, w, I, am, gs, valid = terms(prob)
    occ = occ_mask(prob, occ_mode)
    ca = np.conj(g_ach)[None, None, None, :]
    cs = np.conj(g_asx)[None, None, None, :]
    u = np.where(b1, 1.0 / A, 0.0)
    v = 1.0 / S
    GI = (ca * u + occ * cs * 0.5 * (u - v)).sum(axis=3)                     # [B][P][G]
    GW = (ca * x * u * u + occ * cs * 0.5 * x * (u * u - v * v)).sum(axis=3)
    w3, I3 = w[..., 0], I[..., 0]
    Q = I3 * w3 * GI
    out = {"wtilde": np.conj((M * I3 * GW).sum(axis=0)),
           "I_eps": np.conj((M * w3 * GI).sum(axis=0)),
           "aqsn": np.conj((am[:, :, None] * Q).sum(axis=1))}
    # aqsm enters through its conjugate: vcoul[g] sum over the columns reaching g
    per_col = (prob.aqsntemp[:, None, :] * Q).sum(axis=2) * prob.vcoul[gs][None, :]   # [B][P]
    grad_m = np.zeros_like(prob.aqsmtemp)
    for p in range(prob.ngpown):
        if valid[p]:
            grad_m[:, gs[p]] += per_col[:, p]
    out["aqsm"] = grad_m
    return out


def fast_problems():
    for seed, shape in ((3, (6, 2, 40, 5, 3)), (8, (5, 3, 33, 4, 2)), (13, (7, 2, 24, 6, 4))):
        B, V, G, P, W = shape
        prob = inputs.make_problem(B, V, G, P, W, seed=seed)
        inv = prob.inv_igp_index.copy()
        inv[1] = G                      # the sentinel column
        yield prob.replace(inv_igp_index=inv)


@pytest.mark.parametrize("occ_mode", [0, 1])
def test_forward_partial_fractions_equal_the_oracle(occ_mode):
    for prob in fast_problems():
        b1 = terms(prob)[4]
        assert b1.any() and (~b1).any()          # both branches occur
        got = np.concatenate(forward_partial_fractions(prob, occ_mode))
        ref = np.concatenate(oracle.sigma(prob, occ_mode=occ_mode))
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-12


@pytest.mark.parametrize("occ_mode", [0, 1])
def test_adjoint_partial_fractions_equal_the_oracle(occ_mode):
    for k, prob in enumerate(fast_problems()):
        ga, gs = inputs.cotangents(20 + k, prob.nw)
        got = adjoint_partial_fractions(prob, ga, gs, occ_mode)
        ref = oracle.sigma_adjoint(prob, ga, gs, occ_mode=occ_mode)
        for name in ("wtilde", "I_eps", "aqsm", "aqsn"):
            scale = np.abs(ref[name]).max()
            assert np.abs(got[name] - ref[name]).max() <= 1e-12 * scale, name


def test_a_wrong_identity_is_caught():
    """The test above would see a sign slip in the partial fractions (K/A + K/S)."""
    prob = next(iter(fast_problems()))
    K, A, S, x, b1, *_ = terms(prob)
    ach_terms = np.where(b1, K / A, 0.0)
    wrong = 0.5 * (ach_terms + K / S).sum(axis=(0, 1, 2))
    ref = oracle.sigma(prob)[1]
    assert np.max(np.abs(wrong - ref) / np.abs(ref)) > 1e-3


def test_cancellation_grows_with_x_over_w():
    """Why the kernels bound the partial fractions to x / |w| <= 128: their subtraction
    (K/A - K/S) loses about log2(x / |w|) bits of asxtemp. With every |w| = max x / R the
    numpy form above stays within 1e-13 of the oracle at R = 128 and misses 1e-12 at
    R = 1e6 (the kernels send such warps to the general form)."""
    def worst(R):
        prob = inputs.make_problem(16, 2, 64, 4, 3, seed=5)
        wt = prob.wtilde_array
        wt = (prob.wx_array.max() / R) * np.exp(1j * np.clip(np.angle(wt), -0.2, 0.2))
        prob = prob.replace(wtilde_array=wt)
        got = forward_partial_fractions(prob)[1]
        ref = oracle.sigma(prob)[1]
        return np.max(np.abs(got - ref) / np.abs(ref))
    assert worst(128.0) <= 1e-13
    assert worst(1e6) > 1e-12
