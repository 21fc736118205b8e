"""An independent pure-Python evaluation of the GPP sum, for tiny sizes only.

Test infrastructure: it exists to cross-check the C oracle's loop nest, indexing and
branch selection with code that shares nothing with it (Python ``complex`` arithmetic,
direct division, ``math.fsum`` over the real and imaginary parts). The formulas are the
ones stated in ``gpp_oracle.c`` (paper §II-A loop nest, §III v2 three-way branch).
"""

from __future__ import annotations

import math

LIMITTWO = 0.5 ** 2
LIMITONE = 1.0 / (4.0 * 1.0e-6)
TOL_ZERO = 1.0e-12


def _terms(w: complex, eps: complex, x: float):
    wdiff = x - w
    wdiffr = abs(wdiff) ** 2
    delw = w / wdiff
    delwr = abs(delw) ** 2
    if wdiffr > LIMITTWO and delwr < LIMITONE:
        return delw * eps, w * w * eps / (x * x - w * w)
    if delwr > TOL_ZERO:
        return 0j, -(w * w * eps) * delw / (4.0 * w * w * (delw + 0.5))
    return 0j, 0j


def brute_sigma(prob, occ_mode: int = 0, ch_half: bool = False, sexcut: float = 0.0):
    """(achtemp, asxtemp) as lists of Python complex, one per iw. ``ch_half`` halves every
    sch contribution; ``sexcut > 0`` drops ssx where x < 0 and |ssx| > sexcut |I|."""
    B, V, G, P, W = prob.number_bands, prob.nvband, prob.ncouls, prob.ngpown, prob.nw
    terms_a = [[[], []] for _ in range(W)]
    terms_s = [[[], []] for _ in range(W)]
    for b in range(B):
        occ = 1.0 if occ_mode == 0 else (1.0 if b < V else 0.0)
        for p in range(P):
            k = int(prob.inv_igp_index[p])
            if not 0 <= k <= G:
                continue
            g = int(prob.indinv[k])
            if not 0 <= g < G:
                continue
            for ig in range(G):
                weight = (complex(prob.aqsmtemp[b, g]).conjugate()
                          * complex(prob.aqsntemp[b, ig]) * float(prob.vcoul[g]))
                for iw in range(W):
                    eps = complex(prob.I_eps_array[p, ig])
                    x = float(prob.wx_array[b, iw])
                    sch, ssx = _terms(complex(prob.wtilde_array[p, ig]), eps, x)
                    if sexcut > 0 and x < 0 and abs(ssx) > sexcut * abs(eps):
                        ssx = 0j
                    if ch_half:
                        sch = sch / 2
                    a = weight * sch
                    s = occ * (weight * ssx)
                    terms_a[iw][0].append(a.real)
                    terms_a[iw][1].append(a.imag)
                    terms_s[iw][0].append(s.real)
                    terms_s[iw][1].append(s.imag)
    ach = [complex(math.fsum(t[0]), math.fsum(t[1])) for t in terms_a]
    asx = [complex(math.fsum(t[0]), math.fsum(t[1])) for t in terms_s]
    return ach, asx
