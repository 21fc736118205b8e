"""Plant plausible mistakes in copies of the oracle and check that the pins catch each one.

Every mutant is a text edit of ``oracle/gpp_oracle.c`` (applied at every site where the
text occurs, as a consistent mistake would be) compiled into a temporary library;
the committed oracle is never changed. A mutant that no pin rejects would mean the pins
leave that part of the oracle unchecked.
"""

import os

import pytest

import oracle
import oracle_pins as pins

MUTANTS = {
    "drop vcoul": ("* aqsn[b * G + ig] * vcoul[g];", "* aqsn[b * G + ig];"),
    "drop conj on aqsmtemp": ("cplx mgp = conj(aqsm[b * G + g]);", "cplx mgp = aqsm[b * G + g];"),
    "aqsmtemp by local column": ("cplx mgp = conj(aqsm[b * G + g]);",
                                 "cplx mgp = conj(aqsm[b * G + p]);"),
    "wtilde transposed": ("cplx w = wt[p * G + ig];\n                cplx I = eps[p * G + ig];\n                for (int64_t iw",
                          "cplx w = wt[ig * P + p];\n                cplx I = eps[p * G + ig];\n                for (int64_t iw"),
    "wx transposed": ("gpp_terms_cut(w, I, wx_array[b * W + iw], sexcut, &sch, &ssx, NULL);\n                    cplx a",
                      "gpp_terms_cut(w, I, wx_array[iw * B + b], sexcut, &sch, &ssx, NULL);\n                    cplx a"),
    "branch-2 sign": ("*ssx = -(w2 * I) * delw / (4.0 * w2 * (delw + 0.5));",
                      "*ssx = (w2 * I) * delw / (4.0 * w2 * (delw + 0.5));"),
    "branch-2 half": ("(4.0 * w2 * (delw + 0.5))", "(4.0 * w2 * (delw + 1.0))"),
    "branch-1 denominator": ("*ssx = (w2 * I) / (x * x - w2);", "*ssx = (w2 * I) / (x * x + w2);"),
    "sch uses conj(delw)": ("*sch = delw * I;", "*sch = conj(delw) * I;"),
    "tie goes to branch 1": ("if (wdiffr > LIMITTWO && delwr < LIMITONE)",
                             "if (wdiffr >= LIMITTWO && delwr < LIMITONE)"),
    "limitone dropped": ("if (wdiffr > LIMITTWO && delwr < LIMITONE)", "if (wdiffr > LIMITTWO)"),
    "wdiff sign": ("cplx wdiff = x - w;\n    double wdiffr", "cplx wdiff = w - x;\n    double wdiffr"),
    "occupation ignored": ("double occ = (occ_mode == 1) ? (b < V ? 1.0 : 0.0) : 1.0;\n            cplx mgp",
                           "double occ = 1.0;\n            cplx mgp"),
    "sentinel wraps to column 0": ("if (g < 0 || g >= G) return -1;\n    return g;",
                                   "if (g < 0 || g > G) return -1;\n    return G > 0 ? g % G : -1;"),
    "indinv skipped": ("int64_t g = indinv[k];", "int64_t g = k;"),
    "adjoint dsch/dw": ("*dsch_dw = I * x / (wdiff * wdiff);", "*dsch_dw = I / (wdiff * wdiff);"),
    "adjoint aqsm not conjugate": ("sum_m += ca * n_v * sch + cs * occ * n_v * ssx;",
                                   "sum_m += conj(ca * n_v * sch + cs * occ * n_v * ssx);"),
    "adjoint branch-2 chain": ("*dssx_dw = (-2.0 * I / (d4 * d4)) * ddelw_dw;",
                               "*dssx_dw = (-2.0 * I / (d4 * d4));"),
    "adjoint dssx/dI": ("*dssx_dI = w2 / cden;", "*dssx_dI = w / cden;"),
    "cutoff for any frequency sign": ("sexcut > 0.0 && x < 0.0 && cabs(*ssx)",
                                      "sexcut > 0.0 && cabs(*ssx)"),
    "cutoff without its factor": ("cabs(*ssx) > sexcut * cabs(I)", "cabs(*ssx) > cabs(I)"),
    "cutoff at half its factor": ("cabs(*ssx) > sexcut * cabs(I)", "cabs(*ssx) > 0.5 * sexcut * cabs(I)"),
    "half factor dropped": ("cplx a = (ch_half ? 0.5 : 1.0) * (M * sch);", "cplx a = M * sch;"),
    "half factor on asx too": ("cplx s = occ * (M * ssx);", "cplx s = (ch_half ? 0.5 : 1.0) * occ * (M * ssx);"),
    "adjoint half factor dropped": ("cplx ca = (ch_half ? 0.5 : 1.0) * conj(ga[iw])", "cplx ca = conj(ga[iw])"),
    "adjoint cut derivative kept": ("    if (cut) { /* ssx", "    if (0) { /* ssx"),
    "compensation dropped": ("{ return a->s + a->c; }", "{ return a->s; }"),
    "compensation not accumulated": ("        a->c += (a->s - s) + t;\n    else\n        a->c += (t - s) + a->s;",
                                     "        (void)0;\n    else\n        (void)0;"),
    "compensation branches swapped": ("        a->c += (a->s - s) + t;\n    else\n        a->c += (t - s) + a->s;",
                                      "        a->c += (t - s) + a->s;\n    else\n        a->c += (a->s - s) + t;"),
    "compensation test on signed values": ("if (fabs(a->s) >= fabs(t))", "if (a->s >= t)"),
    "column combine drops the compensation": ("            nsum_add(&tot, part[p * nacc + k].c);\n", ""),
    "column combine uncompensated": ("            nsum_add(&tot, part[p * nacc + k].s);\n            nsum_add(&tot, part[p * nacc + k].c);",
                                     "            tot.s += part[p * nacc + k].s + part[p * nacc + k].c;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(oracle.gpp.SOURCE).read()
    assert src.count(old) >= 1, f"mutation site for {name!r} not found in the oracle"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.compile_oracle(str(path), str(tmp_path / "libmutant.so"))
    mutant = oracle.Oracle(lib)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            fails = pin(mutant)
        except Exception as e:  # a crash or a shape error also rejects the mutant
            fails = [repr(e)]
        if fails:
            caught.append(pin.__name__)
    assert caught, f"no pin rejects the mutant {name!r}"
