"""The FP32-bulk kernel's branch-decision margin, checked on the CPU.

The kernel decides branch 1 (|wdiff|^2 > 1/4) from d = |x - w|^2 - 1/4 evaluated in FP32
(x and Re w each split into an FP32 value and its FP32 residual, x = x_hi + x_lo and
Re w = wr + wr_lo; Ar = (x_hi - wr) + (x_lo - wr_lo), A2 = fma(Ar, Ar, (Im w)^2),
d = A2 - 1/4) and
trusts the sign of d only when |d| exceeds the margin m = 2^-20 (|x| + 252) (formed in FP32
from x_hi); otherwise it recomputes |wdiff|^2 in FP64. The design rests on two claims for the
fast path (x >= 0, Re w >= 0, |w|^2 < 62499, |x| < 1e4):

  * where |d| < 0.1, the FP32 value is within m / 3 of the exact one, so a sign taken
    outside the margin is the exact (and the FP64 kernel's) decision;
  * where |d| >= 0.1, the FP32 sign is always the exact one.

This test evaluates the kernel's FP32 sequence with numpy float32 arithmetic (each
operation rounded to FP32; the fused multiply-add as an FP64 product, exact for FP32
operands, plus one rounding) on seeded samples concentrated at the threshold, and compares
with d computed exactly in rational arithmetic.
"""

from fractions import Fraction

import numpy as np

F32 = np.float32
MARGIN_SCALE = F32(2.0 ** -20)
MARGIN_W = F32(252.0)


def fp32_d(x, wr, wi):
    """The kernel's FP32 d and margin for FP64 inputs."""
    x32, wr32, wi32 = x.astype(F32), wr.astype(F32), wi.astype(F32)
    x_lo = (x - x32.astype(np.float64)).astype(F32)
    wr_lo = (wr - wr32.astype(np.float64)).astype(F32)
    ar = ((x32 - wr32).astype(F32) + (x_lo - wr_lo).astype(F32)).astype(F32)
    wi2 = (wi32 * wi32).astype(F32)
    a2 = (ar.astype(np.float64) * ar.astype(np.float64) + wi2.astype(np.float64)).astype(F32)
    d = (a2 - F32(0.25)).astype(F32)
    m = (MARGIN_SCALE * (np.abs(x32) + MARGIN_W).astype(F32)).astype(F32)
    return d.astype(np.float64), m.astype(np.float64)


def exact_d(x, wr, wi):
    return [float((Fraction(a) - Fraction(b)) ** 2 + Fraction(c) ** 2 - Fraction(1, 4))
            for a, b, c in zip(x.tolist(), wr.tolist(), wi.tolist())]


def fast_path(x, wr, wi):
    w2 = wr * wr + wi * wi
    return (x >= 0) & (x < 1e4) & (wr >= 0) & (w2 > 1e-12) & (w2 < 62499.0)


def test_margin_covers_the_fp32_error_at_the_threshold():
    rng = np.random.Generator(np.random.PCG64(2024))
    n = 40000
    wr = np.concatenate([rng.uniform(0.0, 3.0, n // 2), rng.uniform(0.0, 249.0, n // 2)])
    wi = rng.uniform(-0.499, 0.499, n)
    side = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    x = wr + side * np.sqrt(0.25 - wi * wi) + rng.uniform(-2e-3, 2e-3, n)
    keep = fast_path(x, wr, wi)
    x, wr, wi = x[keep], wr[keep], wi[keep]
    d, m = fp32_d(x, wr, wi)
    de = np.array(exact_d(x, wr, wi))
    assert np.all(np.abs(de) < 0.1)
    err = np.abs(d - de)
    assert np.all(err <= m / 3), float(np.max(err / m))
    # the samples do reach the margin: some fall inside it and go to the FP64 recompute
    assert np.any(np.abs(d) <= m) and np.any(np.abs(d) > m)


def test_far_from_the_threshold_the_fp32_sign_is_exact():
    rng = np.random.Generator(np.random.PCG64(2025))
    n = 40000
    x = np.concatenate([rng.uniform(0.0, 12.0, n // 2), rng.uniform(0.0, 1e4, n // 2)])
    wr = np.concatenate([rng.uniform(0.2, 3.0, n // 2), rng.uniform(0.0, 249.0, n // 2)])
    wi = rng.uniform(-0.6, 0.6, n)
    keep = fast_path(x, wr, wi)
    x, wr, wi = x[keep], wr[keep], wi[keep]
    d, m = fp32_d(x, wr, wi)
    de = np.array(exact_d(x, wr, wi))
    far = np.abs(de) >= 0.1
    assert far.sum() > n // 2
    assert np.all(np.sign(d[far]) == np.sign(de[far]))
    # and wherever the kernel trusts the FP32 sign (outside the margin) it is the exact one
    trusted = np.abs(d) > m
    assert np.all(np.sign(d[trusted]) == np.sign(de[trusted]))


def _rn32(fr: Fraction) -> Fraction:
    """fr rounded to the nearest FP32 value (ties to even), as an exact fraction."""
    f = np.float32(float(fr))
    cands = {f, np.nextafter(f, F32(np.inf)), np.nextafter(f, F32(-np.inf))}
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - fr),
                                     int(np.array(c, dtype=F32).view(np.uint32)) & 1))
    return Fraction(float(best))


def test_bounds_on_x_bracket_x():
    """The per-lane path tests x against the warp's interval through two FMAs on x_hi = RN(x):
    lower bound fma(x_hi, -2^-23, x_hi), upper bound fma(x_hi, 2^-23, x_hi + 2^-126), each
    rounded once to FP32. The upper bound must be >= x everywhere on the fast path
    (0 <= x < 1e4), including x that round to zero or to a subnormal and x next to powers
    of two. The lower bound is compared only with the interval's upper end, max Re w + 1/2
    rounded up (>= 1/2, since Re w >= 0 on the fast path; -inf for a warp without live
    lanes): it must be <= x wherever it reaches 1/2, and it is <= x for every normal x."""
    rng = np.random.Generator(np.random.PCG64(77))
    x = np.concatenate([
        rng.uniform(0.0, 1e4, 3000),
        rng.uniform(0.0, 12.0, 3000),
        np.exp(rng.uniform(np.log(1e-46), np.log(1e-30), 1000)),
        np.array([0.0, 1e-320, 2.0 ** -149, 2.0 ** -126, 1.0, 2.0, 4096.0, 9999.999]),
    ])
    p2 = 2.0 ** rng.integers(-20, 13, 1000).astype(np.float64)
    x = np.concatenate([x, p2 * (1 + rng.uniform(-2e-7, 2e-7, 1000))])
    x = x[(x >= 0) & (x < 1e4)]
    step, tiny = Fraction(2) ** -23, Fraction(2) ** -126
    for xv in x.tolist():
        xh = Fraction(float(np.float32(xv)))
        shifted = _rn32(xh + tiny)   # x_hi + 2^-126, rounded
        lo = _rn32(-xh * step + xh)
        hi = _rn32(xh * step + shifted)
        assert Fraction(xv) <= hi, xv
        assert lo <= Fraction(xv) or (xv < 2.0 ** -126 and lo < Fraction(1, 2)), xv
