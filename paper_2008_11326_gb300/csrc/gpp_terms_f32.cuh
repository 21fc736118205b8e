// The FP32-bulk per-band evaluation (GPP_FP32_BULK), used by the main kernel
// (gpp_batched.cu).
//
// Same decomposition and algebra as the FP64 path (gpp_fwd.cu, gpp_terms_f64.cuh), with the per-term
// complex arithmetic in FP32 on complex64 data: the band-indexed aqsntemp is read from
// its complex64 copy and the gathered weights conj(aqsmtemp) vcoul are rounded once by
// the gather kernel; wtilde and I_eps are read in FP64 once per (igp, ig) pair and rounded
// in registers. FP64 is kept where FP32 would change the answer:
//
//  * Branch decisions. The branch taken at |wdiff|^2 = 1/4 is discontinuous, and FP32
//    rounding of x and w moves |wdiff|^2 by ~1e-7: on the benchmark shape thousands of
//    terms would switch branch, an error of order 1e-4 in the sums. The kernel therefore
//    evaluates d = |wdiff|^2 - 1/4 in FP32 together with a bound m on its rounding error,
//        m = 2^-20 (|x| + 252)  >=  2^-20 (|x| + |Re w| + 2)   (|Re w| < 250 on the fast path),
//    which is at least three times the worst-case error of the FP32 value when |d| < 0.1
//    and |x| < 1e4 (and larger |d| are always decided correctly). If |d| > m the FP32 sign
//    of d is the FP64 decision; otherwise (a fraction ~1e-6 of the terms) the lane
//    recomputes |wdiff|^2 in FP64 exactly as the FP64 kernel does. Every branch decision
//    is therefore the FP64 kernel's.
//  * The pole |wdiff| -> 0. There the FP32 product |wdiff|^2 |x + w|^2 can underflow; for
//    |wdiff|^2 < 2^-30 the branch-2 coefficient 1/|x + w|^2 is taken in FP64.
//  * Accumulation. Terms are summed in FP32 over chunks of kChunk bands, chunk sums are
//    added into compensated (Kahan) FP32 pairs, the pairs are folded into FP64 at the end
//    of every tile, and the block and final reductions are FP64 (gpp_fwd.cu).
//  * Inputs outside the fast path's range (negative frequencies, Re w < 0, |w|^2 outside
//    (1e-12, 62499), |x| >= 1e4) are evaluated by the FP64 general path for the whole warp.
//
// Most terms are far from the threshold: a warp's 32 G-vectors span an interval of Re w,
// and a frequency x more than 1/2 + 2^-20 outside [min Re w, max Re w] is on branch 1 for
// every lane (|wdiff| >= |x - Re w| > 1/2, and 2^-20 exceeds every FP64 rounding of
// |wdiff|^2 near 1/4 for |x| < 1e4), whatever FP32 gives. The kernel forms that interval
// once per (igp, ig) pair with directed rounding and tests x rounded down and up against it
// (two comparisons, the same for the whole warp); such terms skip the decision, the
// margin test, the pole test and both warp votes. When every frequency of a band lies
// beyond the interval on the same side (a per-band range, rounded outwards, against the
// interval: one test), the band takes that path for all frequencies at once.
#pragma once

#include "gpp_device.cuh"

namespace gpp {

constexpr int kChunk = 32;            // bands summed in plain FP32 before a Kahan merge
constexpr float kPoleA2 = 9.313225746154785e-10f;  // 2^-30

__device__ __forceinline__ float rcp_approx_f32(float d) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d));
  return y;
}

__device__ __forceinline__ float2 ldgf2(const float2* p) { return __ldg(p); }

// Selects on the integer pipe. A plain conditional between two floats can be issued as a
// floating-point select, which GB300 executes on its (narrow) FP64 pipe; a bitwise blend
// under an all-ones / all-zeros mask (formed once per term) stays on the integer ALU.
__device__ __forceinline__ unsigned smask(bool c) { return c ? 0xffffffffu : 0u; }
__device__ __forceinline__ float msel(unsigned m, float a, float b) {
  return __uint_as_float((__float_as_uint(a) & m) | (__float_as_uint(b) & ~m));
}

// Per-(igp, ig) constants of the FP32 path.
struct PairF32 {
  float wr, wi, wi2, mw2r, w2i;
  float lo, hi;  // the warp's interval [min Re w - 1/2, max Re w + 1/2], widened by 2^-20
};

// The thread's slots in the FP32 path's shared memory (layout in band_loop_f32): the
// compensated pairs, the FP64 wtilde and the FP64 band table of the instance, the last two
// read only on the rare exact-decision path (kept there rather than in registers).
template <int W>
struct F32Slots {
  static __device__ __forceinline__ float* pair(float* sp, int k) {
    return sp + k * blockDim.x + threadIdx.x;
  }
  static __device__ __forceinline__ double2* w64(float* sp) {
    return reinterpret_cast<double2*>(sp + 2 * 4 * W * blockDim.x) + threadIdx.x;
  }
  static __device__ __forceinline__ const BandEntry** bt64(float* sp) {
    return reinterpret_cast<const BandEntry**>(sp + 2 * 4 * W * blockDim.x + 4 * blockDim.x) +
           threadIdx.x;
  }
  // I w of the thread's G-vector in FP32 (applied to the chunk sums only)
  static __device__ __forceinline__ float2* iw(float* sp) {
    return reinterpret_cast<float2*>(sp + 2 * 4 * W * blockDim.x + 6 * blockDim.x) + threadIdx.x;
  }
};

// Bands [b0, b1) into the chunk sums c. OCC (whether these bands enter asxtemp) is a
// template parameter: a runtime flag in this loop body costs instructions.
template <int W, bool OCC>
__device__ __forceinline__ void bands_f32(int b0, int b1, int G, const float2* __restrict__ an_ptr,
                                          const float2* __restrict__ am_ptr,
                                          const BandEntry32* __restrict__ bt32, float* sp,
                                          const PairF32& q, float (&c)[4 * W]) {
  if (b0 >= b1) return;
  // the next band's aqsntemp and weight are loaded one band ahead (their global-memory
  // latency is the kernel's main stall); inert lanes read a valid element, and their I = 0
  // makes every product vanish
  float2 an_next = ldgf2(an_ptr + static_cast<int64_t>(b0) * G);
  float2 am_next = ldgf2(am_ptr + b0);
#pragma unroll 1
  for (int b = b0; b < b1; ++b) {
    const float2 an = an_next;
    const float2 am = am_next;
    if (b + 1 < b1) {
      an_next = ldgf2(an_ptr + static_cast<int64_t>(b + 1) * G);
      am_next = ldgf2(am_ptr + b + 1);
    }
    // the band sums run on M = am an; band_loop_f32 multiplies them by I w (the same for
    // every band) when it merges a chunk
    const float Kr = fmaf(am.x, an.x, -am.y * an.y);
    const float Ki = fmaf(am.x, an.y, am.y * an.x);
    const float Kwr = -Ki * q.wi, Kwi = Kr * q.wi;
    const float K2r = fmaf(Kr, q.wr, Kwr), K2i = fmaf(Ki, q.wr, Kwi);
    const float P1r = -K2i * q.w2i, P1i = K2r * q.w2i;
    const BandEntry32* e = bt32 + static_cast<int64_t>(b) * W;
    // branch 1 for every lane: K conj(A) / |A|^2 and K2 conj(C) / |C|^2
    auto branch1 = [&](int iw, float x2, float S2, float r, float tr, float ti) {
      const float a1 = S2 * r;
      c[4 * iw + 0] = fmaf(tr, a1, c[4 * iw + 0]);
      c[4 * iw + 1] = fmaf(ti, a1, c[4 * iw + 1]);
      if (OCC) {
        const float Yr = x2 + q.mw2r;
        const float ur = fmaf(K2r, Yr, P1r);
        const float ui = fmaf(K2i, Yr, P1i);
        c[4 * iw + 2] = fmaf(ur, r, c[4 * iw + 2]);
        c[4 * iw + 3] = fmaf(ui, r, c[4 * iw + 3]);
      }
    };
    // the band's frequency range (rounded outwards) rides in the first entry's a.w / b.w
    const float4 e0a = __ldg(&e[0].a);
    const float4 e0b = __ldg(&e[0].b);
    if (e0a.w > q.hi || e0b.w < q.lo) {
      // every frequency of the band outside the warp's interval on the same side
#pragma unroll
      for (int iw = 0; iw < W; ++iw) {
        const float4 ea = iw == 0 ? e0a : __ldg(&e[iw].a);
        const float Ar = ea.x - q.wr;
        const float A2 = fmaf(Ar, Ar, q.wi2);
        const float S2 = fmaf(ea.z, q.wr, A2);
        const float r = rcp_approx_f32(A2 * S2);
        branch1(iw, ea.y, S2, r, fmaf(Kr, Ar, Kwr), fmaf(Ki, Ar, Kwi));
      }
      continue;
    }
#pragma unroll
    for (int iw = 0; iw < W; ++iw) {
      const float4 ea = iw == 0 ? e0a : __ldg(&e[iw].a);
      const float4 eb = iw == 0 ? e0b : __ldg(&e[iw].b);
      const float x = ea.x, x2 = ea.y, x4 = ea.z;
      const float Ar = x - q.wr;
      const float A2 = fmaf(Ar, Ar, q.wi2);
      const float S2 = fmaf(x4, q.wr, A2);
      float r = rcp_approx_f32(A2 * S2);
      const float tr = fmaf(Kr, Ar, Kwr);
      const float ti = fmaf(Ki, Ar, Kwi);
      if (eb.x > q.hi || eb.y < q.lo) {  // x outside the warp's interval
        branch1(iw, x2, S2, r, tr, ti);
        continue;
      }
      float b2 = A2 * r;
      const float d = A2 - 0.25f;
      bool c1 = d > 0.0f;
      const bool near = fabsf(d) <= eb.z;
      const bool pole = A2 < kPoleA2;
      if (__any_sync(0xffffffffu, near || pole)) {
        if (near || pole) {
          const BandEntry* bt64 = *F32Slots<W>::bt64(sp);
          const double x64 = __ldg(&bt64[static_cast<int64_t>(b) * W + iw].lo.x);
          const double2 w64 = *F32Slots<W>::w64(sp);
          const double wi2_64 = w64.y * w64.y;
          if (near) {  // decide exactly as the FP64 kernel
            const double a64 = x64 - w64.x;
            c1 = gt_nonneg(fma(a64, a64, wi2_64), kLimitTwo);
          }
          if (pole) {  // 1/|x + w|^2 in FP64 next to the pole; r only feeds branch 1
            const double s64 = x64 + w64.x;
            b2 = static_cast<float>(rcp_refined(fma(s64, s64, wi2_64)));
            r = 0.0f;
          }
        }
      }
      {  // inside the interval a warp is rarely all on branch 1: no vote, select per lane
        const unsigned m = smask(c1);
        const float a1 = msel(m, S2 * r, 0.0f);
        c[4 * iw + 0] = fmaf(tr, a1, c[4 * iw + 0]);
        c[4 * iw + 1] = fmaf(ti, a1, c[4 * iw + 1]);
        if (OCC) {
          // branch 2: K (-conj(S)/2) / |S|^2 = (Re K Yr - Im K Im w/2, Im K Yr + Re K Im w/2) b2
          const float wih = 0.5f * q.wi;
          const float coef = msel(m, r, b2);
          const float Yr = msel(m, x2, -0.5f * x) + msel(m, q.mw2r, -0.5f * q.wr);
          const float ur = fmaf(msel(m, K2r, Kr), Yr, msel(m, P1r, -Ki * wih));
          const float ui = fmaf(msel(m, K2i, Ki), Yr, msel(m, P1i, Kr * wih));
          c[4 * iw + 2] = fmaf(ur, coef, c[4 * iw + 2]);
          c[4 * iw + 3] = fmaf(ui, coef, c[4 * iw + 3]);
        }
      }
    }
  }
}

// All bands of one (igp, ig) pair into the thread's compensated FP32 pairs hi + lo, which
// live in shared memory (`sp`, layout [2][4W][blockDim.x] floats, then the threads' FP64
// wtilde as double2[blockDim.x], the FP64 band table pointer [blockDim.x] and I w as
// float2[blockDim.x]: touched once per chunk, or only on the rare exact-decision path, they
// would otherwise hold registers through the band loop, and the FP32 path is limited by
// occupancy). Bands are summed in
// FP32 over chunks of kChunk bands and every chunk sum is added to the pair with Kahan's
// compensation.
template <int W>
__device__ __forceinline__ void band_loop_f32(int B, int64_t G, int nocc,
                                              const float2* __restrict__ an_ptr,
                                              const float2* __restrict__ am_ptr,
                                              const BandEntry32* __restrict__ bt32,
                                              const BandEntry* __restrict__ bt64,
                                              double2 w64, double2 I64, bool live,
                                              float* sp) {
  PairF32 q;
  q.wr = static_cast<float>(w64.x);
  q.wi = static_cast<float>(w64.y);
  const float Ir = static_cast<float>(I64.x), Ii = static_cast<float>(I64.y);
  q.wi2 = q.wi * q.wi;
  q.mw2r = -fmaf(q.wr, q.wr, -q.wi2);   // -Re w^2
  q.w2i = 2.0f * q.wr * q.wi;           // Im w^2
  *F32Slots<W>::iw(sp) = make_float2(fmaf(Ir, q.wr, -Ii * q.wi), fmaf(Ir, q.wi, Ii * q.wr));
  *F32Slots<W>::w64(sp) = w64;
  *F32Slots<W>::bt64(sp) = bt64;
  {  // the warp's Re w interval (inert lanes, whose I is 0, left out)
    constexpr double kHalf = 0.5 + 9.5367431640625e-07;  // 1/2 + 2^-20
    float lo = __double2float_rd(w64.x - kHalf), hi = __double2float_ru(w64.x + kHalf);
    if (!live) {
      lo = __int_as_float(0x7f800000);   // +inf
      hi = -lo;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    q.lo = lo;
    q.hi = hi;
  }
#pragma unroll 1
  for (int b0 = 0; b0 < B; b0 += kChunk) {
    float c[4 * W];
#pragma unroll
    for (int k = 0; k < 4 * W; ++k) c[k] = 0.0f;
    const int bend = min(b0 + kChunk, B);
    const int bocc = max(b0, min(nocc, bend));   // bands [b0, bocc) are occupied
    bands_f32<W, true>(b0, bocc, static_cast<int>(G), an_ptr, am_ptr, bt32, sp, q, c);
    if (bocc < bend)
      bands_f32<W, false>(bocc, bend, static_cast<int>(G), an_ptr, am_ptr, bt32, sp, q, c);
    // the chunk sums times I w, merged into the pairs with Kahan's compensation (the pair
    // holds the running sum as hi + lo)
    const float2 Iw = *F32Slots<W>::iw(sp);
#pragma unroll
    for (int k = 0; k < 4 * W; ++k) {
      const float cr = c[k & ~1], ci = c[k | 1];
      const float v = (k & 1) ? fmaf(Iw.x, ci, Iw.y * cr) : fmaf(Iw.x, cr, -Iw.y * ci);
      float& hi = *F32Slots<W>::pair(sp, k);
      float& lo = *F32Slots<W>::pair(sp, 4 * W + k);
      const float y = v + lo;
      const float t = hi + y;
      lo = y - (t - hi);
      hi = t;
    }
  }
}

}  // namespace gpp
