// The FP64 per-band evaluation of the plasmon-pole terms, shared by the FP64 forward
// kernel and the general-input path of the FP32-bulk kernel. The algebra is described at
// the top of gpp_fwd.cu.
#pragma once

#include "gpp_device.cuh"

namespace gpp {

// One band's contribution for the thread's (p, ig) pair, all frequencies.
// FAST: every lane of the warp has 1e-12 < |w|^2 < 62499 and Re w >= 0, and every wx is
// >= 0: branch 1 is exactly |wdiff|^2 > 1/4 and |S|^2 = |A|^2 + 4 x Re(w) has no
// cancellation. Otherwise the general form evaluates both thresholds and forms S directly.
//
// Every term is linear in K = M I w, and I w is the same for all bands of the pair, so
// the band sum runs on M (the weight product) and band_loop multiplies by I w once at the
// end. Per band the caller has formed M, M2 = M w and the cross terms that do not depend on
// the frequency:
//   Mw = (-Im M Im w, Re M Im w)     so that M conj(A) = (Re M Ar + Mw.re, Im M Ar + Mw.im)
//   P1 = (-Im M2 Im w^2, Re M2 Im w^2)  so that M2 conj(C) = (Re M2 Yr + P1.re, Im M2 Yr + P1.im)
//   P2 = Mw / 2 (halved on the integer pipe) so that M (-conj(S)/2) = (Re M Yr + P2.re, Im M Yr + P2.im)
// with Yr = x^2 - Re w^2 (branch 1) or -(x + Re w)/2 (branch 2).
struct BandK {
  double Kr, Ki, K2r, K2i, Kwr, Kwi, P1r, P1i, P2r, P2i;  // M, M2, Mw, P1, P2
};

// sx2 (general form only): sexcut^2 of the screened-exchange cutoff, 0 = off. The cutoff
// drops ssx where x < 0 and |ssx| > sexcut |I|; |ssx| / |I| is |w|^2 / |C| on branch 1 and
// |w| / (2 |S|) on branch 2, compared as |w|^4 / |C|^2 > sx2 and |w|^2 > 4 sx2 |S|^2. (The
// fast path has x >= 0, where the cutoff never applies.)
template <int W, bool FAST, bool OCC>
__device__ __forceinline__ void band_terms(const BandK& k,
                                           const BandEntry* __restrict__ btb, double wr,
                                           double wi2, double wabs2, double mw2r, double wrh,
                                           double sx2, double (&acc)[4 * W]) {
#pragma unroll
  for (int iw = 0; iw < W; ++iw) {
    const double2 xlo = __ldg(&btb[iw].lo);
    const double2 xhi = __ldg(&btb[iw].hi);
    const double x = xlo.x, x2 = xlo.y, x4 = xhi.x, xh = xhi.y;
    const double Ar = x - wr;                 // A = x - w = (Ar, -Im w)
    const double A2 = fma(Ar, Ar, wi2);       // |wdiff|^2
    double S2;
    bool c1, c2;
    if (FAST) {
      S2 = fma(x4, wr, A2);                   // |x + w|^2
      c1 = gt_nonneg(A2, kLimitTwo);
      c2 = true;
    } else {
      const double Sr = x + wr;
      S2 = fma(Sr, Sr, wi2);
      // |delw|^2 = |w|^2 / |wdiff|^2 compared through products (A2 > 0)
      c1 = gt_nonneg(A2, kLimitTwo) && lt_nonneg(wabs2, kLimitOne * A2);
      c2 = gt_nonneg(wabs2, kTolZero * A2);
    }
    const double r = rcp_refined(A2 * S2);
    const double tr = fma(k.Kr, Ar, k.Kwr);
    const double ti = fma(k.Ki, Ar, k.Kwi);
    if (FAST && __all_sync(0xffffffffu, c1)) {
      // the whole warp on branch 1: no selects, and the branch-2 coefficient is not formed
      const double a1 = S2 * r;
      acc[4 * iw + 0] = fma(tr, a1, acc[4 * iw + 0]);
      acc[4 * iw + 1] = fma(ti, a1, acc[4 * iw + 1]);
      if (OCC) {
        const double Yr = x2 + mw2r;
        const double ur = fma(k.K2r, Yr, k.P1r);
        const double ui = fma(k.K2i, Yr, k.P1i);
        acc[4 * iw + 2] = fma(ur, r, acc[4 * iw + 2]);
        acc[4 * iw + 3] = fma(ui, r, acc[4 * iw + 3]);
      }
      continue;
    }
    // achtemp, branch 1 only: K conj(A) / |A|^2
    const double a1 = c1 ? S2 * r : 0.0;
    acc[4 * iw + 0] = fma(tr, a1, acc[4 * iw + 0]);
    acc[4 * iw + 1] = fma(ti, a1, acc[4 * iw + 1]);
    if (OCC) {
      // asxtemp: branch 1 -> K2 conj(C) / |C|^2,  branch 2 -> K (-conj(S)/2) / |S|^2
      const double b2 = A2 * r;
      double coef = c1 ? r : (c2 ? b2 : 0.0);
      if (!FAST) {
        const bool cut = sx2 > 0.0 && x < 0.0 &&
                         (c1 ? gt_nonneg(wabs2 * wabs2 * r, sx2)
                             : gt_nonneg(wabs2, 4.0 * sx2 * S2));
        coef = cut ? 0.0 : coef;
      }
      const double Yr = (c1 ? x2 : xh) + (c1 ? mw2r : wrh);
      const double ur = fma(c1 ? k.K2r : k.Kr, Yr, c1 ? k.P1r : k.P2r);
      const double ui = fma(c1 ? k.K2i : k.Ki, Yr, c1 ? k.P1i : k.P2i);
      acc[4 * iw + 2] = fma(ur, coef, acc[4 * iw + 2]);
      acc[4 * iw + 3] = fma(ui, coef, acc[4 * iw + 3]);
    }
  }
}

// Bands [b0, b1) of the thread's (p, ig) pair. OCC says whether these bands enter asxtemp;
// it is a template parameter because a runtime flag in this loop body costs FP64
// instructions (the compiler schedules the asxtemp terms around it).
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
    BandK k;
    // M = am * an with am = conj(aqsmtemp[b][g]) vcoul[g]; M2 = M w
    k.Kr = fma(am.x, an.x, -am.y * an.y);
    k.Ki = fma(am.x, an.y, am.y * an.x);
    k.Kwr = -k.Ki * wi;
    k.Kwi = k.Kr * wi;
    k.K2r = fma(k.Kr, wr, k.Kwr);   // Re M wr - Im M wi
    k.K2i = fma(k.Ki, wr, k.Kwi);   // Im M wr + Re M wi
    k.P1r = -k.K2i * w2i;
    k.P1i = k.K2r * w2i;
    k.P2r = half_alu(k.Kwr);
    k.P2i = half_alu(k.Kwi);
    band_terms<W, FAST, OCC>(k, bt + static_cast<int64_t>(b) * W, wr, wi2, wabs2, mw2r, wrh, sx2,
                             acc);
  }
}

// All bands of the thread's (p, ig) pair, added to acc: bands [0, nocc) enter both sums,
// the rest only achtemp. The band sums are formed with M and multiplied by Iw = I w here.
// sx2: the screened-exchange cutoff (general form only; see band_terms).
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
