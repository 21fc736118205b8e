"""The restricted finite differences equal the full-problem ones (CPU, oracle only)."""

import numpy as np
import pytest

import fd_restrict
import oracle_pins as pins
from paper_2008_11326_gb300 import inputs


@pytest.mark.parametrize("occ", [0, 1])
def test_restricted_fd_equals_full_fd(orc, occ):
    prob = inputs.make_problem(5, 2, 20, 4, 3, seed=61)
    inv = prob.inv_igp_index.copy()
    inv[2] = inv[1]          # a repeated global column
    inv[3] = prob.ncouls     # a sentinel column
    prob = prob.replace(inv_igp_index=inv)
    ga, gs = inputs.cotangents(3, prob.nw)
    rng = np.random.Generator(np.random.PCG64(2))
    g_rep = int(prob.indinv[inv[1]])
    entries = pins.fd_entries(prob, 3, rng) + [("aqsm", (1, g_rep)), ("wtilde", (3, 4)),
                                               ("aqsn", (4, 7))]
    for kind, idx in entries:
        full = fd_restrict.central_difference(orc, prob, ga, gs, kind, idx, occ_mode=occ, sub=False)
        part = fd_restrict.central_difference(orc, prob, ga, gs, kind, idx, occ_mode=occ)
        assert abs(full - part) <= 1e-7 * max(abs(full), 1e-3), (kind, idx, full, part)


def test_restricted_fd_matches_oracle_adjoint(orc):
    prob = inputs.make_problem(6, 2, 24, 5, 3, seed=62)
    ga, gs = inputs.cotangents(4, prob.nw)
    grads = orc.sigma_adjoint(prob, ga, gs)
    rng = np.random.Generator(np.random.PCG64(3))
    for kind, idx in pins.fd_entries(prob, 4, rng):
        fd = fd_restrict.central_difference(orc, prob, ga, gs, kind, idx)
        assert abs(fd - grads[kind][idx]) <= 1e-6 * max(abs(grads[kind][idx]), 1e-2)
