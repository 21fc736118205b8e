"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each ``pin_*`` function takes a loaded :class:`oracle.Oracle` and returns a list of
failure messages (empty when the pin holds). ``test_oracle_pins.py`` runs them against the
committed oracle; ``test_oracle_mutants.py`` runs them against copies of the oracle with a
planted mistake and checks that some pin fails for every mistake.

Sources of truth:
* hand-derived closed forms at size 1, one hand-derived multi-index case and two exact
  cancellation cases for the compensated summation
  (``tests/golden/closed_forms.json``, derivations inside);
* an independent pure-Python brute force on tiny inputs;
* invariants that follow from the structure of the sum (linearity, conjugation symmetry,
  permutation invariance, additivity over bands and columns, occupation);
* central finite differences of the forward sum, for the adjoint.
"""

from __future__ import annotations

import json
import os
from fractions import Fraction

import numpy as np

import oracle as oracle_pkg
from paper_2008_11326_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "closed_forms.json")

LIMITTWO = 0.25
LIMITONE = 2.5e5
TOL_ZERO = 1e-12


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def cfrac(pair) -> complex:
    return complex(float(Fraction(pair[0])), float(Fraction(pair[1])))


def size1_problem(x, w, I_eps=1 + 0.5j, aqsm=1 + 2j, aqsn=3 - 1j, vcoul=2.0,
                  inv=(0,), nvband=1):
    return inputs.GppProblem(
        number_bands=1, nvband=nvband, ncouls=1, ngpown=1, nw=1,
        aqsmtemp=np.array([[aqsm]], np.complex128),
        aqsntemp=np.array([[aqsn]], np.complex128),
        I_eps_array=np.array([[I_eps]], np.complex128),
        wtilde_array=np.array([[w]], np.complex128),
        vcoul=np.array([vcoul], np.float64),
        inv_igp_index=np.array(inv, np.int32),
        indinv=np.array([0, 1], np.int32),
        wx_array=np.array([[x]], np.float64))


def index_problem():
    B, P, G, W = 2, 2, 3, 2
    aqsm = np.zeros((B, G), np.complex128)
    aqsn = np.zeros((B, G), np.complex128)
    aqsm[1, 2] = 1 + 2j
    aqsn[1, 1] = 3 - 1j
    wt = np.full((P, G), 2 + 0.5j, np.complex128)
    eps = np.ones((P, G), np.complex128)
    wt[0, 1] = 1.0
    eps[0, 1] = 1 + 0.5j
    return inputs.GppProblem(
        number_bands=B, nvband=B, ncouls=G, ngpown=P, nw=W, aqsmtemp=aqsm, aqsntemp=aqsn,
        I_eps_array=eps, wtilde_array=wt, vcoul=np.array([5.0, 7.0, 2.0]),
        inv_igp_index=np.array([0, 2], np.int32), indinv=np.array([2, 1, 0, 3], np.int32),
        wx_array=np.array([[7.0, 9.0], [2.0, 1.25]]))


def _close(got, want, rtol=1e-14, atol=1e-13):
    got = np.asarray(got, np.complex128)
    want = np.asarray(want, np.complex128)
    return bool(np.all(np.abs(got - want) <= atol + rtol * np.abs(want)))


def pin_closed_forms(orc):
    fails = []
    for case in golden()["forward"]:
        prob = size1_problem(float(Fraction(case["x"])), cfrac(case["w"]),
                             inv=tuple(case.get("inv_igp_index", [0])),
                             nvband=case.get("nvband", 1))
        ach, asx = orc.sigma(prob, occ_mode=case.get("occ_mode", 0))
        if not (_close(ach[0], cfrac(case["ach"])) and _close(asx[0], cfrac(case["asx"]))):
            fails.append(f"closed form {case['name']}: got {ach[0]}, {asx[0]}")
    return fails


def pin_physics_closed_forms(orc):
    """The Sigma-code options (half Coulomb-hole factor, screened-exchange cutoff)."""
    fails = []
    for case in golden()["physics"]["cases"]:
        prob = size1_problem(float(Fraction(case["x"])), cfrac(case["w"]))
        ach, asx = orc.sigma(prob, ch_half=case["ch_half"], sexcut=float(Fraction(case["sexcut"])))
        if not (_close(ach[0], cfrac(case["ach"])) and _close(asx[0], cfrac(case["asx"]))):
            fails.append(f"physics closed form {case['name']}: got {ach[0]}, {asx[0]}")
    return fails


def pin_index_case(orc):
    g = golden()["index_case"]
    ach, asx = orc.sigma(index_problem())
    want_a = [cfrac(v) for v in g["ach"]]
    want_s = [cfrac(v) for v in g["asx"]]
    if _close(ach, want_a) and _close(asx, want_s):
        return []
    return [f"index case: got {ach}, {asx}"]


def pin_adjoint_closed_forms(orc):
    fails = []
    for section, x in (("adjoint", 2.0), ("adjoint_branch2", 1.25)):
        g = golden()[section]
        prob = size1_problem(x, 1.0)
        for key, ga, gs in (("re_ach", 1.0, 0.0), ("im_asx", 0.0, 1j)):
            out = orc.sigma_adjoint(prob, np.array([ga]), np.array([gs]))
            for name, want in g[key].items():
                if not _close(out[name][0, 0], cfrac(want)):
                    fails.append(f"{section} {key} d/d{name}: got {out[name][0, 0]}")
    return fails


def pin_adjoint_physics(orc):
    g = golden()["adjoint_physics"]
    prob = size1_problem(-1.1, 1.2)
    fails = []
    for key, ga, gs in (("re_ach", 1.0, 0.0), ("im_asx", 0.0, 1j)):
        out = orc.sigma_adjoint(prob, np.array([ga]), np.array([gs]), ch_half=True, sexcut=4.0)
        for name, want in g[key].items():
            if not _close(out[name][0, 0], cfrac(want)):
                fails.append(f"adjoint_physics {key} d/d{name}: got {out[name][0, 0]}")
    return fails


def summation_problems():
    """The two cancellation cases of the golden file: bands summed within one column, and
    column partials combined across columns."""
    g = golden()["summation"]
    one = np.ones((1, 1), np.complex128)
    bands = g["bands"]
    aqsn = np.array([[complex(float(Fraction(r)), float(Fraction(i)))]
                     for r, i in zip(bands["aqsn_re"], bands["aqsn_im"])], np.complex128)
    B = aqsn.shape[0]
    pb = inputs.GppProblem(
        number_bands=B, nvband=B, ncouls=1, ngpown=1, nw=1,
        aqsmtemp=np.ones((B, 1), np.complex128), aqsntemp=aqsn, I_eps_array=one.copy(),
        wtilde_array=one.copy(), vcoul=np.ones(1), inv_igp_index=np.zeros(1, np.int32),
        indinv=np.array([0, 1], np.int32), wx_array=np.full((B, 1), 3.0))
    cols = g["columns"]
    eps = np.array([[float(Fraction(v))] for v in cols["I_eps"]], np.complex128)
    P = eps.shape[0]
    pc = inputs.GppProblem(
        number_bands=1, nvband=1, ncouls=1, ngpown=P, nw=1, aqsmtemp=one.copy(),
        aqsntemp=np.array([[cfrac(cols["aqsn"])]], np.complex128), I_eps_array=eps,
        wtilde_array=np.ones((P, 1), np.complex128), vcoul=np.ones(1),
        inv_igp_index=np.zeros(P, np.int32), indinv=np.array([0, 1], np.int32),
        wx_array=np.full((1, 1), 3.0))
    return (("bands", pb), ("columns", pc))


def pin_compensated_summation(orc):
    """Exact sums that a plain FP64 running sum gets wrong (every term exact, see the golden
    file): the oracle's compensated summation within a column and across columns."""
    fails = []
    g = golden()["summation"]
    for name, prob in summation_problems():
        ach, asx = orc.sigma(prob)
        want_a, want_s = cfrac(g[name]["ach"]), cfrac(g[name]["asx"])
        if not (ach[0] == want_a and asx[0] == want_s):
            fails.append(f"compensated summation over {name}: got {ach[0]}, {asx[0]}, "
                         f"want {want_a}, {want_s}")
    return fails


def brute_problems():
    out = []
    for seed, (B, V, G, P, W) in enumerate([(3, 2, 12, 3, 3), (4, 1, 16, 5, 2),
                                            (2, 2, 9, 4, 3), (1, 0, 7, 7, 1)]):
        prob = inputs.make_problem(B, V, G, P, W, seed=100 + seed)
        if seed == 1:  # one column on the sentinel, one repeated global column
            inv = prob.inv_igp_index.copy()
            inv[0] = G
            inv[2] = inv[1]
            prob = prob.replace(inv_igp_index=inv)
        if seed == 2:  # frequencies spread over both signs and close to the poles
            wx = np.linspace(-3.0, 3.0, B * W).reshape(B, W)
            prob = prob.replace(wx_array=wx)
        out.append(prob)
    return out


def pin_brute_force(orc):
    fails = []
    for i, prob in enumerate(brute_problems()):
        for occ in (0, 1):
            ach, asx = orc.sigma(prob, occ_mode=occ)
            ba, bs = oracle_pkg.brute_sigma(prob, occ_mode=occ)
            scale = max(np.abs(ba).max(), np.abs(bs).max(), 1e-300)
            err = max(np.abs(ach - np.array(ba)).max(), np.abs(asx - np.array(bs)).max())
            if not err <= 1e-13 * scale:
                fails.append(f"brute force case {i} occ {occ}: err {err:.3e} scale {scale:.3e}")
    # the Sigma-code options, on the case with frequencies of both signs
    prob = brute_problems()[2]
    for ch_half, sexcut in ((True, 0.0), (False, 1.5), (True, 4.0)):
        ach, asx = orc.sigma(prob, ch_half=ch_half, sexcut=sexcut)
        ba, bs = oracle_pkg.brute_sigma(prob, ch_half=ch_half, sexcut=sexcut)
        scale = max(np.abs(ba).max(), np.abs(bs).max(), 1e-300)
        err = max(np.abs(ach - np.array(ba)).max(), np.abs(asx - np.array(bs)).max())
        if not err <= 1e-13 * scale:
            fails.append(f"brute force options {ch_half} {sexcut}: err {err:.3e}")
    return fails


def invariant_problem(seed=11, B=6, V=2, G=48, P=8, W=3):
    return inputs.make_problem(B, V, G, P, W, seed=seed)


def pin_invariants(orc):
    fails = []
    prob = invariant_problem()
    rng = np.random.Generator(np.random.PCG64(99))
    base_a, base_s = orc.sigma(prob)
    scale = max(np.abs(base_a).max(), np.abs(base_s).max())

    def check(name, got, want):
        ga, gs = got
        wa, ws = want
        err = max(np.abs(ga - wa).max(), np.abs(gs - ws).max())
        if not err <= 1e-13 * scale:
            fails.append(f"invariant {name}: err {err:.3e}")

    # linear in aqsntemp
    alpha, beta = 0.7 - 1.3j, -0.4 + 0.9j
    other = prob.aqsntemp[::-1, ::-1].copy()
    oa, os_ = orc.sigma(prob.replace(aqsntemp=other))
    check("linear in aqsntemp",
          orc.sigma(prob.replace(aqsntemp=alpha * prob.aqsntemp + beta * other)),
          (alpha * base_a + beta * oa, alpha * base_s + beta * os_))
    # conjugate-linear in aqsmtemp
    check("conjugate-linear in aqsmtemp", orc.sigma(prob.replace(aqsmtemp=alpha * prob.aqsmtemp)),
          (np.conj(alpha) * base_a, np.conj(alpha) * base_s))
    # vcoul scaling
    check("vcoul scaling", orc.sigma(prob.replace(vcoul=3.0 * prob.vcoul)),
          (3.0 * base_a, 3.0 * base_s))
    # conjugating every complex input conjugates both outputs
    check("conjugation symmetry",
          orc.sigma(prob.replace(aqsmtemp=np.conj(prob.aqsmtemp),
                                 aqsntemp=np.conj(prob.aqsntemp),
                                 I_eps_array=np.conj(prob.I_eps_array),
                                 wtilde_array=np.conj(prob.wtilde_array))),
          (np.conj(base_a), np.conj(base_s)))
    # a consistent permutation of ig over wtilde, I_eps and aqsntemp
    perm = rng.permutation(prob.ncouls)
    check("ig permutation",
          orc.sigma(prob.replace(aqsntemp=prob.aqsntemp[:, perm],
                                 I_eps_array=prob.I_eps_array[:, perm],
                                 wtilde_array=prob.wtilde_array[:, perm])),
          (base_a, base_s))
    # a consistent relabelling of the global columns g over aqsmtemp, vcoul and indinv
    pi = rng.permutation(prob.ncouls)          # old g -> new label pi[g]
    aqsm2 = np.empty_like(prob.aqsmtemp)
    aqsm2[:, pi] = prob.aqsmtemp
    vc2 = np.empty_like(prob.vcoul)
    vc2[pi] = prob.vcoul
    ind2 = prob.indinv.copy()
    ind2[:-1] = pi[prob.indinv[:-1]]
    check("global column relabelling",
          orc.sigma(prob.replace(aqsmtemp=aqsm2, vcoul=vc2, indinv=ind2)), (base_a, base_s))
    # additivity over bands and over columns
    a1, s1 = orc.sigma(prob.bands(slice(0, 2)))
    a2, s2 = orc.sigma(prob.bands(slice(2, None)))
    check("band additivity", (a1 + a2, s1 + s2), (base_a, base_s))
    c1, t1 = orc.sigma(prob.columns(slice(0, 3)))
    c2, t2 = orc.sigma(prob.columns(slice(3, None)))
    check("column additivity", (c1 + c2, t1 + t2), (base_a, base_s))
    # scaling one band's weights by conj(alpha) beta scales that band's contribution
    aqsm3, aqsn3 = prob.aqsmtemp.copy(), prob.aqsntemp.copy()
    aqsm3[1] *= alpha
    aqsn3[1] *= beta
    b1a, b1s = orc.sigma(prob.bands(slice(1, 2)))
    f = np.conj(alpha) * beta
    check("single-band scaling", orc.sigma(prob.replace(aqsmtemp=aqsm3, aqsntemp=aqsn3)),
          (base_a + (f - 1) * b1a, base_s + (f - 1) * b1s))
    # occupation: all bands occupied equals occ_mode 0; no band occupied removes asx only
    check("occupied with nvband = B", orc.sigma(prob.replace(nvband=prob.number_bands), 1),
          (base_a, base_s))
    na, ns = orc.sigma(prob.replace(nvband=0), 1)
    check("occupied with nvband = 0", (na, ns), (base_a, 0 * base_s))
    va, vs = orc.sigma(prob.replace(nvband=2), 1)
    ra, rs = orc.sigma(prob.bands(slice(0, 2)))
    check("occupied bands only in asx", (va, vs), (base_a, rs))
    # a column mapped to the sentinel contributes nothing
    inv = prob.inv_igp_index.copy()
    inv[4] = prob.ncouls
    keep = np.r_[0:4, 5:prob.ngpown]
    check("sentinel column", orc.sigma(prob.replace(inv_igp_index=inv)),
          orc.sigma(prob.columns(keep)))
    return fails


def _loss(orc, prob, ga, gs, **phys):
    ach, asx = orc.sigma(prob, **phys)
    return float(np.sum(np.real(np.conj(ga) * ach)) + np.sum(np.real(np.conj(gs) * asx)))


def _away_from_thresholds(prob, p, ig, margin=0.1, sexcut=0.0):
    w = prob.wtilde_array[p, ig]
    x = prob.wx_array.reshape(-1)
    wdiffr = np.abs(x - w) ** 2
    delwr = np.abs(w) ** 2 / wdiffr
    ok = (np.abs(wdiffr / LIMITTWO - 1) >= margin) & (np.abs(delwr / LIMITONE - 1) >= margin)
    ok &= np.abs(delwr / TOL_ZERO - 1) >= margin
    if sexcut > 0:  # |ssx| / |I| away from the cutoff wherever it applies (x < 0)
        b1 = (wdiffr > LIMITTWO) & (delwr < LIMITONE)
        ratio = np.where(b1, np.abs(w) ** 2 / np.abs(x * x - w * w),
                         np.abs(w) / (2 * np.abs(x + w)))
        ok &= (x >= 0) | (np.abs(ratio / sexcut - 1) >= margin)
    return bool(np.all(ok))


def fd_entries(prob, n_per_kind, rng, sexcut=0.0):
    """(kind, index) pairs; wtilde entries keep every term >= 10% from a threshold."""
    B, G, P = prob.number_bands, prob.ncouls, prob.ngpown
    cols = [int(prob.indinv[k]) for k in prob.inv_igp_index if 0 <= k <= G]
    cols = [g for g in cols if 0 <= g < G]
    out = []
    for kind in ("wtilde", "I_eps", "aqsm", "aqsn"):
        got = 0
        for _ in range(10000):
            if got == n_per_kind:
                break
            if kind in ("wtilde", "I_eps"):
                idx = (int(rng.integers(P)), int(rng.integers(G)))
                if kind == "wtilde" and not _away_from_thresholds(prob, *idx, sexcut=sexcut):
                    continue
            elif kind == "aqsm":
                idx = (int(rng.integers(B)), int(rng.choice(cols)))
            else:
                idx = (int(rng.integers(B)), int(rng.integers(G)))
            out.append((kind, idx))
            got += 1
    return out


_FIELD = {"wtilde": "wtilde_array", "I_eps": "I_eps_array", "aqsm": "aqsmtemp",
          "aqsn": "aqsntemp"}


def central_difference(orc, prob, ga, gs, kind, idx, h=1e-6, **phys):
    field = _FIELD[kind]
    parts = []
    for step in (h, 1j * h):
        vals = []
        for sgn in (1, -1):
            arr = getattr(prob, field).copy()
            arr[idx] += sgn * step
            vals.append(_loss(orc, prob.replace(**{field: arr}), ga, gs, **phys))
        parts.append((vals[0] - vals[1]) / (2 * h))
    return complex(parts[0], parts[1])


def fd_problems():
    """A config-shaped instance, and one whose frequencies sit among the wtilde values so
    that many terms take branch 2 (|wdiff| <= 1/2)."""
    a = inputs.make_problem(4, 2, 16, 4, 3, seed=21)
    b = inputs.make_problem(5, 2, 12, 3, 3, seed=22)
    b = b.replace(wx_array=np.linspace(0.3, 2.9, 15).reshape(5, 3))
    return a, b


def pin_adjoint_fd(orc, n_per_kind=4):
    fails = []
    for k, prob in enumerate(fd_problems()):
        ga, gs = inputs.cotangents(3, prob.nw)
        grads = orc.sigma_adjoint(prob, ga, gs)
        rng = np.random.Generator(np.random.PCG64(5 + k))
        for kind, idx in fd_entries(prob, n_per_kind, rng):
            fd = central_difference(orc, prob, ga, gs, kind, idx)
            adj = grads[kind][idx]
            if not abs(fd - adj) <= 1e-6 * max(abs(adj), 1e-2):
                fails.append(f"adjoint vs FD problem {k} d/d{kind}{idx}: adj {adj} fd {fd}")
    # the Sigma-code options, on frequencies of both signs (some terms cut, some kept)
    prob = fd_problems()[1]
    prob = prob.replace(wx_array=prob.wx_array - 1.6)
    phys = dict(ch_half=True, sexcut=1.5)
    ga, gs = inputs.cotangents(4, prob.nw)
    grads = orc.sigma_adjoint(prob, ga, gs, **phys)
    rng = np.random.Generator(np.random.PCG64(8))
    for kind, idx in fd_entries(prob, n_per_kind, rng, sexcut=phys["sexcut"]):
        fd = central_difference(orc, prob, ga, gs, kind, idx, **phys)
        adj = grads[kind][idx]
        if not abs(fd - adj) <= 1e-6 * max(abs(adj), 1e-2):
            fails.append(f"adjoint vs FD with options d/d{kind}{idx}: adj {adj} fd {fd}")
    return fails


ALL_PINS = (pin_closed_forms, pin_physics_closed_forms, pin_index_case,
            pin_compensated_summation,
            pin_adjoint_closed_forms, pin_adjoint_physics, pin_brute_force, pin_invariants,
            pin_adjoint_fd)
