"""The kernels' fast path decides branch 1 from |wdiff|^2 alone; checked against the
oracle's three-way branch on the CPU.

On the fast path (x >= 0, Re w >= 0, 1e-12 < |w|^2 < 62499) the paper's branch (§III v2 on
squared moduli, §III v3) reduces to |wdiff|^2 > 1/4: there |delw|^2 = |w|^2 / |wdiff|^2 is
below 62499 / (1/4) < LIMITONE whenever |wdiff|^2 > 1/4, and above 1e-12 / (1/4) > TOL_ZERO
otherwise, so branch 3 never occurs and branch 1 needs no |delw|^2 test. The FP64 and
FP32-bulk kernels rely on this (their general path keeps the full test). This test samples
the fast path, densely at |wdiff|^2 = 1/4 and at its |w| bounds, and asks the oracle.
"""

import numpy as np

import oracle


def kernel_fast_branch(w, x):
    return 1 if abs(x - w) ** 2 > 0.25 else 2


def samples(rng, n):
    out = []
    # at the threshold |x - w| = 1/2
    wr = rng.uniform(0.0, 249.0, n)
    wi = rng.uniform(-0.49, 0.49, n)
    side = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    x = wr + side * np.sqrt(0.25 - wi * wi) + rng.uniform(-1e-6, 1e-6, n)
    out += list(zip(wr + 1j * wi, x))
    # |w| near the fast path's upper bound (|w|^2 just under 62499), x far and near
    ang = rng.uniform(-1e-3, 1e-3, n)
    r = np.sqrt(62499.0) * (1.0 - rng.uniform(1e-9, 1e-6, n))
    w = r * np.exp(1j * ang)
    x = np.where(rng.random(n) < 0.5, w.real + rng.uniform(-3.0, 3.0, n), rng.uniform(0, 1e4, n))
    out += list(zip(w, np.abs(x)))
    # |w| near the lower bound (|w|^2 just over 1e-12), x within 1/2 of it and beyond
    w = (1e-6 * (1.0 + rng.uniform(1e-6, 1.0, n))) * np.exp(1j * rng.uniform(-1.5, 1.5, n))
    x = rng.uniform(0.0, 1.0, n)
    out += list(zip(w, x))
    return [(w, x) for w, x in out if x >= 0 and w.real >= 0 and 1e-12 < abs(w) ** 2 < 62499.0
            and x != w]


def test_fast_path_branch_equals_the_three_way_branch():
    rng = np.random.Generator(np.random.PCG64(77))
    cases = samples(rng, 20000)
    assert len(cases) > 50000
    seen = set()
    for w, x in cases:
        b = oracle.branch(complex(w), float(x))
        assert b == kernel_fast_branch(complex(w), float(x)), (w, x, b)
        seen.add(b)
    assert seen == {1, 2}
