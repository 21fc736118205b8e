// The FP64 per-band evaluation of the plasmon-pole terms, shared by the FP64 forward
// kernel and the general-input path of the FP32-bulk kernel. The algebra is described at
// the top of gpp_fwd.cu.
#pragma once

#include "gpp_device.cuh"

namespace gpp {

// The fast path: every lane of the warp has 1e-12 < |w|^2 < 62499 and Re w >= 0, and
// every wx is >= 0. There branch 1 is exactly |wdiff|^2 > 1/4, branch 3 never occurs and the
// screened-exchange cutoff (x < 0 only) never applies, and the terms are taken in partial
// fractions. With the weight M, A = x - w and S = x + w:
//   achtemp, branch 1:   M/A
//   asxtemp, branch 1:   M w / (A S) = (M/A - M/S) / 2
//   asxtemp, branch 2:   -M / (2 S)
// so over a set of bands asxtemp = (achtemp - sum M/S) / 2, whatever the branches. A term
// costs two complex reciprocals, 1/A = conj(A)/|A|^2 and 1/S = conj(S)/|S|^2 (one FP64
// reciprocal each), and two complex multiply-adds; the asxtemp side needs no branch and no
// per-band M w products. (The subtraction gives up at most a few bits of FP64 where |M/A|
// exceeds the asxtemp term.) Every term is linear in K = M I w and I w is the same for all
// bands of a (p, ig) pair, so the band sums run on M and band_loop multiplies by I w at
// the end. The caller passes M and Mw = (-Im M Im w, Re M Im w), so that
//   M conj(A) = (Re M Ar + Mw.re, Im M Ar + Mw.im),  M conj(S) = (Re M Sr - Mw.re, Im M Sr - Mw.im)
// with Ar = x - Re w, Sr = x + Re w. acc[4 iw + 0, 1] collects the branch-1 sum of M/A and,
// with OCC, acc[4 iw + 2, 3] the sum of M/S.
template <int W, bool OCC>
__device__ __forceinline__ void band_terms_fast(double Kr, double Ki, double Kwr, double Kwi,
                                                const BandEntry* __restrict__ btb, double wr,
                                                double wi2, double (&acc)[4 * W]) {
#pragma unroll
  for (int iw = 0; iw < W; ++iw) {
    const double x = __ldg(&btb[iw].lo.x);
    const double Ar = x - wr;
    const double A2 = fma(Ar, Ar, wi2);           // |wdiff|^2
    const double ra = rcp_refined(A2);
    const double a1 = gt_nonneg(A2, kLimitTwo) ? ra : 0.0;
    acc[4 * iw + 0] = fma(fma(Kr, Ar, Kwr), a1, acc[4 * iw + 0]);
    acc[4 * iw + 1] = fma(fma(Ki, Ar, Kwi), a1, acc[4 * iw + 1]);
    if (OCC) {
      const double Sr = x + wr;
      const double S2 = fma(Sr, Sr, wi2);         // |x + w|^2 >= |w|^2 > 1e-12
      const double rs = rcp_refined(S2);
      acc[4 * iw + 2] = fma(fma(Kr, Sr, -Kwr), rs, acc[4 * iw + 2]);
      acc[4 * iw + 3] = fma(fma(Ki, Sr, -Kwi), rs, acc[4 * iw + 3]);
    }
  }
}

// The general form, for warps outside the fast path's conditions: both thresholds, the
// screened-exchange cutoff, and S formed directly. One band's contribution for the thread's
// (p, ig) pair, all frequencies. Per band the caller has formed M, M2 = M w and the cross
// terms that do not depend on the frequency:
//   Mw = (-Im M Im w, Re M Im w)     so that M conj(A) = (Re M Ar + Mw.re, Im M Ar + Mw.im)
//   P1 = (-Im M2 Im w^2, Re M2 Im w^2)  so that M2 conj(C) = (Re M2 Yr + P1.re, Im M2 Yr + P1.im)
//   P2 = Mw / 2 (halved on the integer pipe) so that M (-conj(S)/2) = (Re M Yr + P2.re, Im M Yr + P2.im)
// with Yr = x^2 - Re w^2 (branch 1) or -(x + Re w)/2 (branch 2); one reciprocal
// r = 1/(|A|^2 |S|^2) serves the three denominators (gpp_fwd.cu).
struct BandK {
  double Kr, Ki, K2r, K2i, Kwr, Kwi, P1r, P1i, P2r, P2i;  // M, M2, Mw, P1, P2
};

// sx2: sexcut^2 of the screened-exchange cutoff, 0 = off. The cutoff drops ssx where x < 0
// and |ssx| > sexcut |I|; |ssx| / |I| is |w|^2 / |C| on branch 1 and |w| / (2 |S|) on branch
// 2, compared as |w|^4 / |C|^2 > sx2 and |w|^2 > 4 sx2 |S|^2.
template <int W, bool OCC>
__device__ __forceinline__ void band_terms_general(const BandK& k,
                                                   const BandEntry* __restrict__ btb,
                                                   double wr, double wi2, double wabs2,
                                                   double mw2r, double wrh, double sx2,
                                                   double (&acc)[4 * W]) {
#pragma unroll
  for (int iw = 0; iw < W; ++iw) {
    const double2 xlo = __ldg(&btb[iw].lo);
    const double x = xlo.x, x2 = xlo.y, xh = __ldg(&btb[iw].hi.y);
    const double Ar = x - wr;                 // A = x - w = (Ar, -Im w)
    const double A2 = fma(Ar, Ar, wi2);       // |wdiff|^2
    const double Sr = x + wr;
    const double S2 = fma(Sr, Sr, wi2);
    // |delw|^2 = |w|^2 / |wdiff|^2 compared through products (A2 > 0)
    const bool c1 = gt_nonneg(A2, kLimitTwo) && lt_nonneg(wabs2, kLimitOne * A2);
    const bool c2 = gt_nonneg(wabs2, kTolZero * A2);
    const double r = rcp_refined(A2 * S2);
    const double tr = fma(k.Kr, Ar, k.Kwr);
    const double ti = fma(k.Ki, Ar, k.Kwi);
    // achtemp, branch 1 only: K conj(A) / |A|^2
    const double a1 = c1 ? S2 * r : 0.0;
    acc[4 * iw + 0] = fma(tr, a1, acc[4 * iw + 0]);
    acc[4 * iw + 1] = fma(ti, a1, acc[4 * iw + 1]);
    if (OCC) {
      // asxtemp: branch 1 -> K2 conj(C) / |C|^2,  branch 2 -> K (-conj(S)/2) / |S|^2
      const double b2 = A2 * r;
      double coef = c1 ? r : (c2 ? b2 : 0.0);
      const bool cut = sx2 > 0.0 && x < 0.0 &&
                       (c1 ? gt_nonneg(wabs2 * wabs2 * r, sx2)
                           : gt_nonneg(wabs2, 4.0 * sx2 * S2));
      coef = cut ? 0.0 : coef;
      const double Yr = (c1 ? x2 : xh) + (c1 ? mw2r : wrh);
      const double ur = fma(c1 ? k.K2r : k.Kr, Yr, c1 ? k.P1r : k.P2r);
      const double ui = fma(c1 ? k.K2i : k.Ki, Yr, c1 ? k.P1i : k.P2i);
      acc[4 * iw + 2] = fma(ur, coef, acc[4 * iw + 2]);
      acc[4 * iw + 3] = fma(ui, coef, acc[4 * iw + 3]);
    }
  }
}

// Bands [b0, b1) of the thread's (p, ig) pair, by the fast or the general form. OCC says
// whether these bands enter asxtemp; it is a template parameter because a runtime flag in
// this loop body costs FP64 instructions (the compiler schedules the asxtemp terms around
// it). With FAST, acc[4 iw + 2, 3] collects sum M/S (see band_terms_fast).
template <int W, bool FAST, bool OCC>
__device__ __forceinline__ void band_range(int b0, int b1, int64_t G,
                                           const double2* __restrict__ an_ptr,
                                           const double2* __restrict__ am_ptr,
                                           const BandEntry* __restrict__ bt, bool live, double wr,
                                           double wi, double wi2, double wabs2, double mw2r,
                                           double w2i, double wrh, double sx2,
                                           double (&acc)[4 * W]) {
#pragma unroll 1
  for (int b = b0; b < b1; ++b) {
    const double2 an = live ? ldg2(an_ptr + static_cast<int64_t>(b) * G) : make_double2(0.0, 0.0);
    const double2 am = ldg2(am_ptr + b);
    // M = am * an with am = conj(aqsmtemp[b][g]) vcoul[g], and Mw
    const double Kr = fma(am.x, an.x, -am.y * an.y);
    const double Ki = fma(am.x, an.y, am.y * an.x);
    const double Kwr = -Ki * wi, Kwi = Kr * wi;
    if (FAST) {
      band_terms_fast<W, OCC>(Kr, Ki, Kwr, Kwi, bt + static_cast<int64_t>(b) * W, wr, wi2, acc);
      continue;
    }
    BandK k;
    k.Kr = Kr;
    k.Ki = Ki;
    k.Kwr = Kwr;
    k.Kwi = Kwi;
    k.K2r = fma(Kr, wr, Kwr);   // M2 = M w: Re M wr - Im M wi
    k.K2i = fma(Ki, wr, Kwi);   //           Im M wr + Re M wi
    k.P1r = -k.K2i * w2i;
    k.P1i = k.K2r * w2i;
    k.P2r = half_alu(Kwr);
    k.P2i = half_alu(Kwi);
    band_terms_general<W, OCC>(k, bt + static_cast<int64_t>(b) * W, wr, wi2, wabs2, mw2r, wrh,
                               sx2, acc);
  }
}

// All bands of the thread's (p, ig) pair, added to acc: bands [0, nocc) enter both sums,
// the rest only achtemp. The band sums are formed with M and multiplied by Iw = I w here.
// sx2: the screened-exchange cutoff (general form only; see band_terms_general).
template <int W, bool FAST>
__device__ __forceinline__ void band_loop(int B, int64_t G, int nocc,
                                          const double2* __restrict__ an_ptr,
                                          const double2* __restrict__ am_ptr,
                                          const BandEntry* __restrict__ bt, bool live,
                                          double wr, double wi, double Iwr, double Iwi,
                                          double sx2, double (&acc)[4 * W]) {
  const double wi2 = wi * wi;
  const double wabs2 = fma(wr, wr, wi2);
  const double mw2r = -fma(wr, wr, -wi2);   // -Re w^2
  const double w2i = 2.0 * wr * wi;         // Im w^2
  const double wrh = -0.5 * wr;
  double t[4 * W];
#pragma unroll
  for (int k = 0; k < 4 * W; ++k) t[k] = 0.0;
  band_range<W, FAST, true>(0, nocc, G, an_ptr, am_ptr, bt, live, wr, wi, wi2, wabs2, mw2r, w2i,
                            wrh, sx2, t);
  if (FAST) {   // the occupied bands' asxtemp: (their achtemp - sum M/S) / 2
#pragma unroll
    for (int iw = 0; iw < W; ++iw) {
      t[4 * iw + 2] = 0.5 * (t[4 * iw + 0] - t[4 * iw + 2]);
      t[4 * iw + 3] = 0.5 * (t[4 * iw + 1] - t[4 * iw + 3]);
    }
  }
  if (nocc < B)
    band_range<W, FAST, false>(nocc, B, G, an_ptr, am_ptr, bt, live, wr, wi, wi2, wabs2, mw2r,
                               w2i, wrh, sx2, t);
#pragma unroll
  for (int k = 0; k < 2 * W; ++k) {   // acc += Iw t, per complex value
    const double tr = t[2 * k], ti = t[2 * k + 1];
    acc[2 * k] = fma(Iwr, tr, fma(-Iwi, ti, acc[2 * k]));
    acc[2 * k + 1] = fma(Iwr, ti, fma(Iwi, tr, acc[2 * k + 1]));
  }
}

}  // namespace gpp
