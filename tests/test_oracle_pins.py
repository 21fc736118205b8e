"""The CPU oracle against hand-derived closed forms, brute force, invariants and finite
differences (see ``oracle_pins.py`` for what each pin rests on)."""

import numpy as np
import pytest

import oracle_pins as pins
from paper_2008_11326_gb300 import inputs


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    fails = pin(orc)
    assert not fails, "\n".join(fails)


def test_branch_selection(orc):
    # paper Sec. III v2: the three-way branch, taken on squared moduli (Sec. III v3)
    assert orc.branch(1.0, 2.0) == 1
    assert orc.branch(1.0, 1.25) == 2          # |wdiff| <= 1/2
    assert orc.branch(1.0, 1.5) == 2           # tie at LIMITTWO falls through
    assert orc.branch(1000.0, 1000.75) == 2    # |delw| >= 500
    assert orc.branch(1e-8, 0.1) == 3          # |delw|^2 <= TOL_ZERO
    assert orc.branch(1.0 + 1.0j, 3.0) == 1


def test_thread_count_does_not_change_bits(orc):
    prob = inputs.config("tiny")
    a1, s1 = orc.sigma(prob, nthreads=1)
    a4, s4 = orc.sigma(prob, nthreads=4)
    assert np.array_equal(a1, a4) and np.array_equal(s1, s4)


def test_empty_sizes(orc):
    for B, G, P, W in [(0, 8, 2, 3), (3, 8, 0, 3), (3, 8, 2, 0)]:
        prob = inputs.make_problem(B, 2, G, P, W, seed=1)
        a, s = orc.sigma(prob)
        assert a.shape == (W,) and np.all(a == 0) and np.all(s == 0)


def test_adjoint_grads_zero_on_unreached_columns(orc):
    prob = inputs.make_problem(3, 2, 10, 2, 2, seed=8)
    ga, gs = inputs.cotangents(3, prob.nw)
    out = orc.sigma_adjoint(prob, ga, gs)
    cols = {int(prob.indinv[k]) for k in prob.inv_igp_index}
    for g in range(prob.ncouls):
        if g not in cols:
            assert np.all(out["aqsm"][:, g] == 0)
