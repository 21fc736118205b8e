"""Central finite differences of the oracle's loss on sub-problems that keep exactly the
terms depending on one input entry.

The loss is L = sum_iw Re(conj(g_ach) ach + conj(g_asx) asx). Perturbing one entry of
wtilde / I_eps (p, ig), aqsntemp (b, ig) or aqsmtemp (b, g) changes only the terms that
read it; every other term cancels in L(z + h) - L(z - h). The sub-problem holds those
terms (plus terms whose weight is exactly zero), so its central difference equals the full
problem's, with far less rounding. Only index bookkeeping happens here; all arithmetic of
the sum is the oracle's.
"""

from __future__ import annotations

import numpy as np

from paper_2008_11326_gb300 import inputs

_FIELD = {"wtilde": "wtilde_array", "I_eps": "I_eps_array", "aqsm": "aqsmtemp",
          "aqsn": "aqsntemp"}


def _column(prob, p):
    k = int(prob.inv_igp_index[p])
    if not 0 <= k <= prob.ncouls:
        return -1
    g = int(prob.indinv[k])
    return g if 0 <= g < prob.ncouls else -1


def restrict(prob, kind, idx):
    """Sub-problem holding every term that depends on entry ``idx`` of input ``kind``.
    Returns (sub_problem, index of the entry inside it)."""
    B, G, P, W = prob.number_bands, prob.ncouls, prob.ngpown, prob.nw
    if kind in ("wtilde", "I_eps"):
        p, ig = idx
        g = _column(prob, p)
        aqsm = np.zeros((B, 2), np.complex128)
        aqsn = np.zeros((B, 2), np.complex128)
        aqsn[:, 0] = prob.aqsntemp[:, ig]
        vc = np.array([1.0, 1.0])
        if g >= 0:
            aqsm[:, 1] = prob.aqsmtemp[:, g]
            vc[1] = prob.vcoul[g]
        sub = inputs.GppProblem(
            B, prob.nvband, 2, 1, W, aqsm, aqsn,
            np.array([[prob.I_eps_array[p, ig], 0.0]]),
            np.array([[prob.wtilde_array[p, ig], 0.5 + 1.0j]]),
            vc, np.array([0], np.int32), np.array([1 if g >= 0 else 2, 0, 2], np.int32),
            prob.wx_array.copy())
        return sub, (0, 0)
    if kind == "aqsn":
        b, ig = idx
        Gs = 1 + P
        aqsm = np.zeros((1, Gs), np.complex128)
        aqsn = np.zeros((1, Gs), np.complex128)
        aqsn[0, 0] = prob.aqsntemp[b, ig]
        vc = np.ones(Gs)
        wt = np.full((P, Gs), 0.5 + 1.0j, np.complex128)
        eps = np.zeros((P, Gs), np.complex128)
        wt[:, 0] = prob.wtilde_array[:, ig]
        eps[:, 0] = prob.I_eps_array[:, ig]
        indinv = np.empty(Gs + 1, np.int32)
        indinv[:P] = np.arange(1, P + 1)
        indinv[P:] = Gs
        for p in range(P):
            g = _column(prob, p)
            if g >= 0:
                aqsm[0, 1 + p] = prob.aqsmtemp[b, g]
                vc[1 + p] = prob.vcoul[g]
            else:
                indinv[p] = Gs  # contributes nothing, as in the full problem
        sub = inputs.GppProblem(1, prob.nvband - b if prob.nvband > b else 0, Gs, P, W, aqsm,
                                aqsn, eps, wt, vc, np.arange(P, dtype=np.int32), indinv,
                                prob.wx_array[b:b + 1].copy())
        return sub, (0, 0)
    if kind == "aqsm":
        b, g = idx
        cols = [p for p in range(P) if _column(prob, p) == g]
        sub = inputs.GppProblem(
            1, prob.nvband - b if prob.nvband > b else 0, G, len(cols), W,
            prob.aqsmtemp[b:b + 1].copy(), prob.aqsntemp[b:b + 1].copy(),
            prob.I_eps_array[cols].copy(), prob.wtilde_array[cols].copy(), prob.vcoul.copy(),
            prob.inv_igp_index[cols].copy(), prob.indinv.copy(), prob.wx_array[b:b + 1].copy())
        return sub, (0, g)
    raise ValueError(kind)


def loss(orc, prob, g_ach, g_asx, occ_mode=0):
    ach, asx = orc.sigma(prob, occ_mode=occ_mode)
    return float(np.sum(np.real(np.conj(g_ach) * ach)) + np.sum(np.real(np.conj(g_asx) * asx)))


def central_difference(orc, prob, g_ach, g_asx, kind, idx, h=1e-6, occ_mode=0, sub=True):
    """(dL/dRe z + i dL/dIm z) at entry ``idx`` of ``kind`` by central differences."""
    if sub:
        prob, idx = restrict(prob, kind, idx)
    field = _FIELD[kind]
    parts = []
    for step in (h, 1j * h):
        vals = []
        for sgn in (1, -1):
            arr = getattr(prob, field).copy()
            arr[idx] += sgn * step
            vals.append(loss(orc, prob.replace(**{field: arr}), g_ach, g_asx, occ_mode))
        parts.append((vals[0] - vals[1]) / (2 * h))
    return complex(parts[0], parts[1])
