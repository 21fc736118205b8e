/*
 * Plain FP64 CPU oracle for the General Plasmon Pole (GPP) self-energy summation.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline /
 * reference legs of the benchmark load this library. The product (the CUDA library and
 * its Python binding) never links, imports or calls it, and the two share no code.
 *
 * What is computed. The loop nest is the paper's (§II-A): for every band, every local
 * column igp, every G-vector ig and every frequency iw, load wtilde_array, aqsntemp and
 * the inverse dielectric matrix, form wdiff and delw, choose sch and ssx by the three-way
 * branch of §III v2 (predicates on squared moduli, §III v3) and accumulate into
 * achtemp[iw] and asxtemp[iw]. The paper names the branch constants and says "calculate
 * sch, ssx" without printing them; the formulas below are the Hybertsen-Louie generalised
 * plasmon-pole terms of BerkeleyGW's Sigma module (the code the paper takes the kernel
 * from), written out as mathematics:
 *
 *   g      = indinv[inv_igp_index[p]]          (the global column of local column p;
 *                                               g outside [0, G) contributes nothing)
 *   M      = conj(aqsmtemp[b][g]) * aqsntemp[b][ig] * vcoul[g]
 *   x      = wx_array[b][iw]   (real)          w = wtilde_array[p][ig]   I = I_eps_array[p][ig]
 *   wdiff  = x - w             wdiffr = |wdiff|^2
 *   delw   = w / wdiff         delwr  = |delw|^2
 *   if wdiffr > LIMITTWO and delwr < LIMITONE:  sch = delw * I
 *                                               ssx = w^2 I / (x^2 - w^2)
 *   else if delwr > TOL_ZERO:                   sch = 0
 *                                               ssx = -(w^2 I) delw / (4 w^2 (delw + 1/2))
 *   else:                                       sch = 0,  ssx = 0
 *   achtemp[iw] += M * sch       asxtemp[iw] += occ(b) * M * ssx
 *
 * occ(b) = 1 for every band (occ_mode 0, "all bands", as the paper's loop nest sums every
 * band) or [b < nvband] (occ_mode 1, occupied bands only).
 *
 * Two options from the Sigma code the kernel sits in (BerkeleyGW; not in the paper's loop
 * nest, off by default):
 *   ch_half != 0: achtemp[iw] += (1/2) M sch  (the factor 1/2 of the Coulomb-hole sum);
 *   sexcut > 0:   a term with x < 0 and |ssx| > sexcut |I| takes ssx = 0 (the screened-
 *                 exchange cutoff; the comparison is strict).
 *
 * The constants are a reading (the paper does not print their values): LIMITTWO = 0.5^2,
 * LIMITONE = 1 / (4 * 1e-6), TOL_ZERO = 1e-12, all compared against squared moduli with
 * strict inequalities, so a tie falls through to the next branch.
 *
 * Arithmetic: C99 double complex with the written divisions (no reciprocal tricks, no
 * algebraic rearrangement). Build with -O2 -ffp-contract=off and no fast-math. The
 * reduction is the plain sum, evaluated with Neumaier-compensated summation: one running
 * compensated sum per local column p over (b, ig), then a compensated combine in p order.
 * The result does not depend on the thread count.
 *
 * Parity note: whether these branch formulas and constants are exactly what the paper's
 * kernel evaluated is unpinned; the paper prints neither. Everything else (loop nest,
 * branch structure, indexing) is pinned by the closed-form, invariant and brute-force tests.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* complex.h defines I as the imaginary unit; the paper's I (the inverse dielectric
 * matrix element) takes the name here, and the unit is spelled _Complex_I. */
#undef I

static int thread_count(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

#define LIMITTWO 0.25
#define LIMITONE (1.0 / (4.0 * 1.0e-6))
#define TOL_ZERO 1.0e-12

typedef double complex cplx;

/* Neumaier's compensated running sum (Neumaier 1974). */
typedef struct {
    double s, c;
} nsum;

static inline void nsum_add(nsum *a, double t)
{
    double s = a->s + t;
    if (fabs(a->s) >= fabs(t))
        a->c += (a->s - s) + t;
    else
        a->c += (t - s) + a->s;
    a->s = s;
}

static inline double nsum_value(const nsum *a) { return a->s + a->c; }

/* Global column of local column p, or -1 when the column contributes nothing. */
static inline int64_t global_column(int64_t p, int64_t G, const int32_t *inv_igp_index,
                                    const int32_t *indinv)
{
    int64_t k = inv_igp_index[p];
    if (k < 0 || k > G) return -1;
    int64_t g = indinv[k];
    if (g < 0 || g >= G) return -1;
    return g;
}

/* The plasmon-pole terms for one (w, I, x): returns the branch taken (1, 2 or 3). With
 * sexcut > 0, ssx is set to zero (and *cut to 1, when cut is not NULL) for x < 0 and
 * |ssx| > sexcut |I|. */
static int gpp_terms_cut(cplx w, cplx I, double x, double sexcut, cplx *sch, cplx *ssx,
                         int *cut);

static int gpp_terms(cplx w, cplx I, double x, cplx *sch, cplx *ssx)
{
    cplx wdiff = x - w;
    double wdiffr = creal(wdiff) * creal(wdiff) + cimag(wdiff) * cimag(wdiff);
    cplx delw = w / wdiff;
    double delwr = creal(delw) * creal(delw) + cimag(delw) * cimag(delw);
    if (wdiffr > LIMITTWO && delwr < LIMITONE) {
        cplx w2 = w * w;
        *sch = delw * I;
        *ssx = (w2 * I) / (x * x - w2);
        return 1;
    } else if (delwr > TOL_ZERO) {
        cplx w2 = w * w;
        *sch = 0.0;
        *ssx = -(w2 * I) * delw / (4.0 * w2 * (delw + 0.5));
        return 2;
    }
    *sch = 0.0;
    *ssx = 0.0;
    return 3;
}

static int gpp_terms_cut(cplx w, cplx I, double x, double sexcut, cplx *sch, cplx *ssx,
                         int *cut)
{
    int br = gpp_terms(w, I, x, sch, ssx);
    int c = sexcut > 0.0 && x < 0.0 && cabs(*ssx) > sexcut * cabs(I);
    if (c) *ssx = 0.0;
    if (cut) *cut = c;
    return br;
}

static int check_sizes(int64_t B, int64_t V, int64_t G, int64_t P, int64_t W)
{
    if (B < 0 || V < 0 || G < 0 || P < 0 || W < 0) return -2;
    return 0;
}

/*
 * Forward sum. All complex arrays are interleaved (re, im) doubles, row-major:
 * aqsmtemp, aqsntemp [B][G]; I_eps_array, wtilde_array [P][G]; vcoul [G];
 * inv_igp_index [P]; indinv [G+1]; wx_array [B][W]. Outputs achtemp, asxtemp [W] complex.
 * ch_half and sexcut as in the header (0 and 0.0: the paper's sum). nthreads <= 0 uses the
 * OpenMP default. Returns 0, or -2 for negative sizes.
 */
int oracle_gpp_sigma(int64_t B, int64_t V, int64_t G, int64_t P, int64_t W, int occ_mode,
                     int ch_half, double sexcut,
                     const double *aqsmtemp, const double *aqsntemp,
                     const double *I_eps_array, const double *wtilde_array,
                     const double *vcoul, const int32_t *inv_igp_index,
                     const int32_t *indinv, const double *wx_array,
                     double *achtemp, double *asxtemp, int nthreads)
{
    if (check_sizes(B, V, G, P, W)) return -2;
    const cplx *aqsm = (const cplx *)aqsmtemp;
    const cplx *aqsn = (const cplx *)aqsntemp;
    const cplx *eps = (const cplx *)I_eps_array;
    const cplx *wt = (const cplx *)wtilde_array;
    /* per column p: W ach sums (re, im) then W asx sums (re, im) */
    int64_t nacc = 4 * W;
    nsum *part = (nsum *)calloc((size_t)(P > 0 ? P : 1) * (size_t)(nacc > 0 ? nacc : 1),
                                sizeof(nsum));
    if (!part) return -1;
    int nt = thread_count(nthreads);
    (void)nt;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t p = 0; p < P; ++p) {
        int64_t g = global_column(p, G, inv_igp_index, indinv);
        if (g < 0) continue;
        nsum *acc = part + p * nacc;
        for (int64_t b = 0; b < B; ++b) {
            double occ = (occ_mode == 1) ? (b < V ? 1.0 : 0.0) : 1.0;
            cplx mgp = conj(aqsm[b * G + g]);
            for (int64_t ig = 0; ig < G; ++ig) {
                cplx M = mgp * aqsn[b * G + ig] * vcoul[g];
                cplx w = wt[p * G + ig];
                cplx I = eps[p * G + ig];
                for (int64_t iw = 0; iw < W; ++iw) {
                    cplx sch, ssx;
                    gpp_terms_cut(w, I, wx_array[b * W + iw], sexcut, &sch, &ssx, NULL);
                    cplx a = (ch_half ? 0.5 : 1.0) * (M * sch);
                    cplx s = occ * (M * ssx);
                    nsum_add(&acc[2 * iw + 0], creal(a));
                    nsum_add(&acc[2 * iw + 1], cimag(a));
                    nsum_add(&acc[2 * W + 2 * iw + 0], creal(s));
                    nsum_add(&acc[2 * W + 2 * iw + 1], cimag(s));
                }
            }
        }
    }
    for (int64_t k = 0; k < nacc; ++k) {
        nsum tot = {0.0, 0.0};
        for (int64_t p = 0; p < P; ++p) {
            nsum_add(&tot, part[p * nacc + k].s);
            nsum_add(&tot, part[p * nacc + k].c);
        }
        double v = nsum_value(&tot);
        if (k < 2 * W)
            achtemp[k] = v;
        else
            asxtemp[k - 2 * W] = v;
    }
    free(part);
    return 0;
}

/*
 * The plasmon-pole terms and their derivatives with respect to w and I, from the written
 * formulas. Inside each branch the terms are holomorphic in w and I; the branch
 * predicates are locally constant, so they contribute no derivative.
 *   branch 1: d sch/dw = I x / (x - w)^2          d ssx/dw = 2 w x^2 I / (x^2 - w^2)^2
 *             d sch/dI = delw                      d ssx/dI = w^2 / (x^2 - w^2)
 *   branch 2: d delw/dw = x / (x - w)^2,  d ssx/d delw = -2 I / (4 delw + 2)^2
 *             d ssx/dw = (d ssx/d delw)(d delw/dw) d ssx/dI = -(w^2) delw / (4 w^2 (delw + 1/2))
 * and both ssx derivatives are zero where the screened-exchange cutoff sets ssx to zero.
 */
static void gpp_terms_grad(cplx w, cplx I, double x, double sexcut, cplx *sch, cplx *ssx,
                           cplx *dsch_dw, cplx *dssx_dw, cplx *dsch_dI, cplx *dssx_dI)
{
    int cut;
    int br = gpp_terms_cut(w, I, x, sexcut, sch, ssx, &cut);
    cplx wdiff = x - w;
    if (br == 1) {
        cplx w2 = w * w;
        cplx cden = x * x - w2;
        *dsch_dw = I * x / (wdiff * wdiff);
        *dssx_dw = 2.0 * w * (x * x) * I / (cden * cden);
        *dsch_dI = w / wdiff;
        *dssx_dI = w2 / cden;
    } else if (br == 2) {
        cplx w2 = w * w;
        cplx delw = w / wdiff;
        cplx d4 = 4.0 * delw + 2.0;
        cplx ddelw_dw = x / (wdiff * wdiff);
        *dsch_dw = 0.0;
        *dssx_dw = (-2.0 * I / (d4 * d4)) * ddelw_dw;
        *dsch_dI = 0.0;
        *dssx_dI = -w2 * delw / (4.0 * w2 * (delw + 0.5));
    } else {
        *dsch_dw = 0.0;
        *dssx_dw = 0.0;
        *dsch_dI = 0.0;
        *dssx_dI = 0.0;
    }
    if (cut) { /* ssx is identically zero where the cutoff holds (a locally constant test) */
        *dssx_dw = 0.0;
        *dssx_dI = 0.0;
    }
}

/*
 * Reference adjoint. Given the cotangents of the outputs in the PyTorch convention for
 * complex tensors (g = dL/dRe + i dL/dIm, so that dL = Re(conj(g) dy)), returns
 *   dL/dRe z + i dL/dIm z
 * for z in wtilde_array, I_eps_array, aqsmtemp, aqsntemp. With c = conj(g) and F the
 * per-term contribution, a holomorphic input gets conj(c dF/dz) and aqsmtemp (which
 * enters through its conjugate) gets c dF/d conj(aqsmtemp). Terms are recomputed, not
 * stored. Any output pointer may be NULL (that gradient is skipped). Sums are plain FP64
 * in a fixed loop order. Pass 1 runs over columns p (wtilde, I_eps); pass 2 over bands b
 * (aqsntemp, aqsmtemp; entries of aqsmtemp not reached by any column are zero).
 */
int oracle_gpp_sigma_adjoint(int64_t B, int64_t V, int64_t G, int64_t P, int64_t W,
                             int occ_mode, int ch_half, double sexcut,
                             const double *aqsmtemp, const double *aqsntemp,
                             const double *I_eps_array, const double *wtilde_array,
                             const double *vcoul, const int32_t *inv_igp_index,
                             const int32_t *indinv, const double *wx_array,
                             const double *g_ach, const double *g_asx,
                             double *grad_wtilde, double *grad_I_eps,
                             double *grad_aqsmtemp, double *grad_aqsntemp, int nthreads)
{
    if (check_sizes(B, V, G, P, W)) return -2;
    const cplx *aqsm = (const cplx *)aqsmtemp;
    const cplx *aqsn = (const cplx *)aqsntemp;
    const cplx *eps = (const cplx *)I_eps_array;
    const cplx *wt = (const cplx *)wtilde_array;
    const cplx *ga = (const cplx *)g_ach;
    const cplx *gs = (const cplx *)g_asx;
    cplx *dw_out = (cplx *)grad_wtilde;
    cplx *dI_out = (cplx *)grad_I_eps;
    cplx *dm_out = (cplx *)grad_aqsmtemp;
    cplx *dn_out = (cplx *)grad_aqsntemp;
    int nt = thread_count(nthreads);
    (void)nt;
    if (dw_out || dI_out) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
        for (int64_t p = 0; p < P; ++p) {
            int64_t g = global_column(p, G, inv_igp_index, indinv);
            for (int64_t ig = 0; ig < G; ++ig) {
                if (dw_out) dw_out[p * G + ig] = 0.0;
                if (dI_out) dI_out[p * G + ig] = 0.0;
            }
            if (g < 0) continue;
            for (int64_t ig = 0; ig < G; ++ig) {
                cplx w = wt[p * G + ig];
                cplx I = eps[p * G + ig];
                cplx sum_w = 0.0, sum_I = 0.0;
                for (int64_t b = 0; b < B; ++b) {
                    double occ = (occ_mode == 1) ? (b < V ? 1.0 : 0.0) : 1.0;
                    cplx M = conj(aqsm[b * G + g]) * aqsn[b * G + ig] * vcoul[g];
                    for (int64_t iw = 0; iw < W; ++iw) {
                        cplx sch, ssx, dsch_dw, dssx_dw, dsch_dI, dssx_dI;
                        gpp_terms_grad(w, I, wx_array[b * W + iw], sexcut, &sch, &ssx,
                                       &dsch_dw, &dssx_dw, &dsch_dI, &dssx_dI);
                        cplx ca = (ch_half ? 0.5 : 1.0) * conj(ga[iw]), cs = conj(gs[iw]);
                        sum_w += conj(ca * M * dsch_dw + cs * occ * M * dssx_dw);
                        sum_I += conj(ca * M * dsch_dI + cs * occ * M * dssx_dI);
                    }
                }
                if (dw_out) dw_out[p * G + ig] = sum_w;
                if (dI_out) dI_out[p * G + ig] = sum_I;
            }
        }
    }
    if (dm_out || dn_out) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
        for (int64_t b = 0; b < B; ++b) {
            double occ = (occ_mode == 1) ? (b < V ? 1.0 : 0.0) : 1.0;
            for (int64_t ig = 0; ig < G; ++ig) {
                if (dm_out) dm_out[b * G + ig] = 0.0;
                if (dn_out) dn_out[b * G + ig] = 0.0;
            }
            for (int64_t p = 0; p < P; ++p) {
                int64_t g = global_column(p, G, inv_igp_index, indinv);
                if (g < 0) continue;
                cplx m_conj_v = conj(aqsm[b * G + g]) * vcoul[g];
                cplx sum_m = 0.0;
                for (int64_t ig = 0; ig < G; ++ig) {
                    cplx w = wt[p * G + ig];
                    cplx I = eps[p * G + ig];
                    cplx n_v = aqsn[b * G + ig] * vcoul[g];
                    cplx sum_n = 0.0;
                    for (int64_t iw = 0; iw < W; ++iw) {
                        cplx sch, ssx;
                        gpp_terms_cut(w, I, wx_array[b * W + iw], sexcut, &sch, &ssx, NULL);
                        cplx ca = (ch_half ? 0.5 : 1.0) * conj(ga[iw]), cs = conj(gs[iw]);
                        /* F = conj(aqsm) aqsn vcoul (sch | occ ssx) */
                        sum_n += conj(ca * m_conj_v * sch + cs * occ * m_conj_v * ssx);
                        sum_m += ca * n_v * sch + cs * occ * n_v * ssx;
                    }
                    if (dn_out) dn_out[b * G + ig] += sum_n;
                }
                if (dm_out) dm_out[b * G + g] += sum_m;
            }
        }
    }
    return 0;
}

/* Branch taken by one term (1, 2 or 3), for tests that steer inputs into a branch. */
int oracle_gpp_branch(double w_re, double w_im, double x)
{
    cplx sch, ssx;
    return gpp_terms(w_re + _Complex_I * w_im, 0.0, x, &sch, &ssx);
}
