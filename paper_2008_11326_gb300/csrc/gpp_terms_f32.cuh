// The FP32-bulk per-band evaluation (GPP_FP32_BULK), used by the main kernel
// (gpp_batched.cu).
//
// Same decomposition and algebra as the FP64 path (gpp_fwd.cu, gpp_terms_f64.cuh), with the
// per-term complex arithmetic in FP32 on complex64 data: the band-indexed aqsntemp is read
// from its complex64 copy and the gathered weights conj(aqsmtemp) vcoul are rounded once by
// the gather kernel; wtilde and I_eps are read in FP64 once per (igp, ig) pair. FP64 (or
// FP32 pairs carrying FP64 information) is kept where FP32 would change the answer or lose
// accuracy that does not average out:
//
//  * Branch decisions. The branch taken at |wdiff|^2 = 1/4 is discontinuous, and FP32
//    rounding moves |wdiff|^2 by ~1e-7: on the benchmark shape thousands of terms would
//    switch branch, an error of order 1e-4 in the sums. The kernel evaluates
//    d = |wdiff|^2 - 1/4 in FP32 together with a bound m on its rounding error,
//        m = 2^-20 (|x| + 252)  >=  2^-20 (|x| + |Re w| + 2)   (|Re w| < 250 on the fast path),
//    which is at least three times the worst-case error of the FP32 value when |d| < 0.1
//    and |x| < 1e4 (and larger |d| are always decided correctly). If |d| > m the FP32 sign
//    of d is the FP64 decision; otherwise (a fraction ~1e-6 of the terms) the lane
//    recomputes |wdiff|^2 in FP64 exactly as the FP64 kernel does. Every branch decision
//    is therefore the FP64 kernel's.
//  * The difference x - Re w. Rounding x and Re w to FP32 separately moves wdiff by up to
//    2^-24 (|x| + |Re w|), which relative to |wdiff| (>= 1/2 on branch 1) is up to ~30
//    FP32 units for the benchmark's frequencies, and the same rounding of x (once per band)
//    or of Re w (once per G-vector) is shared by many terms. Both carry their FP32 residual
//    (x = x_hi + x_lo from the band table, Re w = wr + wr_lo per thread), and
//    Ar = (x_hi - wr) + (x_lo - wr_lo) is accurate to a few units of Ar itself. S = x + w
//    and Re C = Ar Sr + (Im w)^2 (C = x^2 - w^2 = A S) are formed from Ar and Sr, without the
//    cancellation of x^2 - Re w^2.
//  * The pole |wdiff| -> 0. There the FP32 product |wdiff|^2 |x + w|^2 can underflow; for
//    |wdiff|^2 < 2^-30 the branch-2 coefficient 1/|x + w|^2 is taken in FP64.
//  * Accumulation. Terms are summed in FP32 over chunks of kChunk bands (the rounding error
//    of a running FP32 sum grows with the number of terms in it), every chunk sum is added
//    to a running FP32 sum with Kahan's compensation (the compensation carried into the next
//    chunk's sum), the two forming a compensated pair, and once per (igp, ig) pair the pair is
//    multiplied by I w in double-FP32 arithmetic (I w formed in FP64) and added into the
//    thread's compensated tile sums; the block and final reductions are compensated pairs
//    and FP64 (gpp_batched.cu).
//  * Inputs outside the fast path's range (negative frequencies, Re w < 0, |w|^2 outside
//    (1e-12, 62499), |x| >= 1e4) are evaluated by the FP64 general path for the whole warp.
//
// Most terms are far from the threshold: a warp's 32 G-vectors span an interval of Re w,
// and a frequency x more than 1/2 + 2^-20 outside [min Re w, max Re w] is on branch 1 for
// every lane (|wdiff| >= |x - Re w| > 1/2, and 2^-20 exceeds every FP64 rounding of
// |wdiff|^2 near 1/4 for |x| < 1e4), whatever FP32 gives. The kernel forms that interval
// once per (igp, ig) pair with directed rounding and tests lower and upper bounds on x
// against it (x_hi (1 -/+ 2^-23), formed in two FMAs; two comparisons, the same for the
// whole warp); such terms skip the decision, the
// margin test, the pole test and both warp votes. When every frequency of a band lies
// beyond the interval on the same side (a per-band range, rounded outwards, against the
// interval: one test), the band takes that path for all frequencies at once.
#pragma once

#include "gpp_device.cuh"

namespace gpp {

#ifndef GPP_F32_CHUNK
#define GPP_F32_CHUNK 16
#endif
constexpr int kChunk = GPP_F32_CHUNK;  // bands summed in plain FP32 before a Kahan merge
constexpr float kPoleA2 = 9.313225746154785e-10f;  // 2^-30

__device__ __forceinline__ float rcp_approx_f32(float d) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d));
#ifdef GPP_F32_RCP_NEWTON
  y = fmaf(y, fmaf(-d, y, 1.0f), y);
#endif
  return y;
}

__device__ __forceinline__ float2 ldgf2(const float2* p) { return __ldg(p); }

// L1 eviction priorities for the band loop's read-only loads. Each band streams a new
// aqsntemp row through L1 (a CTA's 1 KB per band, read by its four warps within a short
// window: evict first), while every CTA on the SM walks the same small band table (80 bytes
// per band at nw = 3: evict last), which the streaming rows would otherwise push out.
__device__ __forceinline__ float2 ld_stream_f2(const float2* p) {
  float2 v;
  asm("ld.global.nc.L1::evict_first.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_keep_f4(const float4* p) {
  float4 v;
  asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}

// Selects on the integer pipe. A plain conditional between two floats can be issued as a
// floating-point select, which GB300 executes on its (narrow) FP64 pipe; a bitwise blend
// under an all-ones / all-zeros mask (formed once per term) stays on the integer ALU.
__device__ __forceinline__ unsigned smask(bool c) { return c ? 0xffffffffu : 0u; }
__device__ __forceinline__ float msel(unsigned m, float a, float b) {
  return __uint_as_float((__float_as_uint(a) & m) | (__float_as_uint(b) & ~m));
}

// Per-(igp, ig) constants of the FP32 path.
struct PairF32 {
  float wr, wr_lo, wi, wi2, w2i;  // Re w = wr + wr_lo; Im w; (Im w)^2; Im w^2
  float lo, hi;  // the warp's interval [min Re w - 1/2, max Re w + 1/2], widened by 2^-20
};

// The thread's slots in the FP32 path's dynamic shared memory: the band sums' compensated
// pairs (4W hi values then 4W lo values), each stored as float4 with a stride of blockDim.x
// (a thread's four consecutive values in one 16-byte access, conflict-free across a warp),
// then the thread's FP64 wtilde (double2), read only on the rare exact-decision path and
// at the end of a pair's band loop. Kept here rather than in registers, which bound the
// kernel's occupancy. (The tile sums' compensated pairs, touched once per pair, live in
// the thread's local memory: in shared memory they would take the L1 capacity that the
// band loop's aqsntemp loads hit in.)
template <int W>
struct F32Slots {
  static constexpr int kFloats = 8 * W + 4;  // per thread
  // band pairs: quads [0, W) hold hi[4q .. 4q + 3] (the four values of frequency q: Re ach,
  // Im ach, Re asx, Im asx), quads [W, 2W) lo
  static __device__ __forceinline__ float4* band4(float* sp, int q) {
    return reinterpret_cast<float4*>(sp) + q * blockDim.x + threadIdx.x;
  }
  static __device__ __forceinline__ double2* w64(float* sp) {
    return reinterpret_cast<double2*>(sp + 8 * W * blockDim.x) + threadIdx.x;
  }
};

// Index of value (component k, frequency iw) in the chunk sums: frequency pairs first (the
// two frequencies of a pair adjacent, pair-aligned, for the paired FP32 instructions), then
// the last frequency when W is odd.
template <int W>
__host__ __device__ constexpr int ci(int k, int iw) {
  return iw < 2 * (W / 2) ? (k * (W / 2) + iw / 2) * 2 + (iw & 1) : 8 * (W / 2) + k;
}

__device__ __forceinline__ float& quad_elem(float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// The rare exact path of a term: with `near`, the branch decided from |wdiff|^2 in FP64
// exactly as the FP64 kernel does; with `pole` (|wdiff|^2 < 2^-30), the branch-2
// coefficient 1/|x + w|^2 in FP64 (r, which only feeds branch 1, is then 0).
template <int W>
__device__ __forceinline__ void exact_decision(const BandEntry* bt64, int k, float* sp, bool near,
                                            bool pole, bool& c1, float& b2, float& r) {
  const double x64 = __ldg(&bt64[k].lo.x);
  const double2 w64 = *F32Slots<W>::w64(sp);
  const double wi2_64 = w64.y * w64.y;
  if (near) {
    const double a64 = x64 - w64.x;
    c1 = gt_nonneg(fma(a64, a64, wi2_64), kLimitTwo);
  }
  if (pole) {
    const double s64 = x64 + w64.x;
    b2 = static_cast<float>(rcp_refined(fma(s64, s64, wi2_64)));
    r = 0.0f;
  }
}

// Bands [b0, b1) into the chunk sums c. OCC (whether these bands enter asxtemp) is a
// template parameter: a runtime flag in this loop body costs instructions. `bt64` (the FP64
// band table, for the rare exact path) is read from shared memory.
template <int W, bool OCC>
__device__ __forceinline__ void bands_f32(int b0, int b1, int G, const float2* __restrict__ an_ptr,
                                          const float2* __restrict__ am_ptr,
                                          const float4* __restrict__ bt32,
                                          const BandEntry* const* s_bt64, float* sp,
                                          const PairF32& q, float (&c)[4 * W]) {
  constexpr int NQ = f32_half_quads(W), FB = f32_band_quads(W);
  if (b0 >= b1) return;
  // the next band's aqsntemp and weight are loaded one band ahead (their global-memory
  // latency is the kernel's main stall); inert lanes read a valid element, and their I = 0
  // makes every product vanish. (Loading the band table's block one band ahead as well
  // needs registers the 72-register budget does not have: the spills cost more, 124 ms
  // against 104 ms on the benchmark instance.)
  float2 an_next = ld_stream_f2(an_ptr + static_cast<int64_t>(b0) * G);
  float2 am_next = ldgf2(am_ptr + b0);
#pragma unroll 4
  for (int b = b0; b < b1; ++b) {
    const float2 an = an_next;
    const float2 am = am_next;
    if (b + 1 < b1) {
      an_next = ld_stream_f2(an_ptr + static_cast<int64_t>(b + 1) * G);
      am_next = ldgf2(am_ptr + b + 1);
    }
    // the band sums run on M = am an; the caller multiplies them by I w (the same for
    // every band) once the pair's bands are done
    const float Kr = fmaf(am.x, an.x, -am.y * an.y);
    const float Ki = fmaf(am.x, an.y, am.y * an.x);
    const float Kwr = -Ki * q.wi, Kwi = Kr * q.wi;
    const float K2r = fmaf(Kr, q.wr, Kwr), K2i = fmaf(Ki, q.wr, Kwi);
    const float P1r = -K2i * q.w2i, P1i = K2r * q.w2i;
    // the far-path block: x_hi[], the band's lowest frequency; x_lo[], its highest
    const float4* e = bt32 + static_cast<int64_t>(b) * FB;
    float4 hq[NQ], lq[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      hq[k] = ld_keep_f4(&e[k]);
      lq[k] = ld_keep_f4(&e[NQ + k]);
    }
    auto xh = [&](int i) -> float { return quad_elem(hq[i >> 2], i & 3); };
    auto xl = [&](int i) -> float { return quad_elem(lq[i >> 2], i & 3); };
    // branch 1 for every lane: M conj(A) / |A|^2 and M w conj(C) / |C|^2
    auto branch1 = [&](int iw, float Ar, float Sr, float S2, float r, float tr, float ti) {
      const float a1 = S2 * r;
      c[ci<W>(0, iw)] = fmaf(tr, a1, c[ci<W>(0, iw)]);
      c[ci<W>(1, iw)] = fmaf(ti, a1, c[ci<W>(1, iw)]);
      if (OCC) {
        const float Yr = fmaf(Ar, Sr, q.wi2);  // Re C = Ar Sr + (Im w)^2
        const float ur = fmaf(K2r, Yr, P1r);
        const float ui = fmaf(K2i, Yr, P1i);
        c[ci<W>(2, iw)] = fmaf(ur, r, c[ci<W>(2, iw)]);
        c[ci<W>(3, iw)] = fmaf(ui, r, c[ci<W>(3, iw)]);
      }
    };
    if (xh(W) > q.hi || xl(W) < q.lo) {
      // every frequency of the band outside the warp's interval on the same side
      // frequency pairs in GB300's paired FP32 instructions (FADD2 / FMUL2 / FFMA2: two
      // FP32 operations per lane per instruction, each rounded as its scalar form, so the
      // result is the scalar path's bit for bit); the chunk sums of a pair are adjacent
      // (ci), the per-band and per-thread operands are duplicated into pairs
      const float2 KR2 = make_float2(Kr, Kr), KI2 = make_float2(Ki, Ki);
      const float2 KWR2 = make_float2(Kwr, Kwr), KWI2 = make_float2(Kwi, Kwi);
      const float2 K2R2 = make_float2(K2r, K2r), K2I2 = make_float2(K2i, K2i);
      const float2 P1R2 = make_float2(P1r, P1r), P1I2 = make_float2(P1i, P1i);
      const float2 NWR2 = make_float2(-q.wr, -q.wr), NWRL2 = make_float2(-q.wr_lo, -q.wr_lo);
      const float2 WR2 = make_float2(q.wr, q.wr), WI22 = make_float2(q.wi2, q.wi2);
#pragma unroll
      for (int iw = 0; iw + 1 < W; iw += 2) {
        const float2 XH = make_float2(xh(iw), xh(iw + 1));
        const float2 XL = make_float2(xl(iw), xl(iw + 1));
        const float2 AR = __fadd2_rn(__fadd2_rn(XH, NWR2), __fadd2_rn(XL, NWRL2));
        const float2 SR = __fadd2_rn(XH, WR2);
        const float2 A2 = __ffma2_rn(AR, AR, WI22);
        const float2 S2 = __ffma2_rn(SR, SR, WI22);
        const float2 DEN = __fmul2_rn(A2, S2);
        const float2 R = make_float2(rcp_approx_f32(DEN.x), rcp_approx_f32(DEN.y));
        const float2 A1 = __fmul2_rn(S2, R);
        const float2 TR = __ffma2_rn(KR2, AR, KWR2);
        const float2 TI = __ffma2_rn(KI2, AR, KWI2);
        float2* c2 = reinterpret_cast<float2*>(c);
        c2[ci<W>(0, iw) / 2] = __ffma2_rn(TR, A1, c2[ci<W>(0, iw) / 2]);
        c2[ci<W>(1, iw) / 2] = __ffma2_rn(TI, A1, c2[ci<W>(1, iw) / 2]);
        if (OCC) {
          const float2 YR = __ffma2_rn(AR, SR, WI22);
          const float2 UR = __ffma2_rn(K2R2, YR, P1R2);
          const float2 UI = __ffma2_rn(K2I2, YR, P1I2);
          c2[ci<W>(2, iw) / 2] = __ffma2_rn(UR, R, c2[ci<W>(2, iw) / 2]);
          c2[ci<W>(3, iw) / 2] = __ffma2_rn(UI, R, c2[ci<W>(3, iw) / 2]);
        }
      }
      if (W & 1) {
        const int iw = W - 1;
        const float Ar = (xh(iw) - q.wr) + (xl(iw) - q.wr_lo);
        const float Sr = xh(iw) + q.wr;
        const float A2 = fmaf(Ar, Ar, q.wi2);
        const float S2 = fmaf(Sr, Sr, q.wi2);
        const float r = rcp_approx_f32(A2 * S2);
        branch1(iw, Ar, Sr, S2, r, fmaf(Kr, Ar, Kwr), fmaf(Ki, Ar, Kwi));
      }
      continue;
    }
#pragma unroll
    for (int iw = 0; iw < W; ++iw) {
      // bounds on x (x >= 0 on this path): x_hi (1 -/+ 2^-23) lie beyond the FP32
      // neighbours of x_hi, and FLT_MIN covers an x that rounds to zero or a subnormal (the
      // lower bound exceeds such an x only below 1/2, and it is compared only with the
      // interval's upper end, >= 1/2 or -inf)
      const float xrd = fmaf(xh(iw), -0x1p-23f, xh(iw));
      const float xru = fmaf(xh(iw), 0x1p-23f, xh(iw) + 0x1p-126f);
      const float Ar = (xh(iw) - q.wr) + (xl(iw) - q.wr_lo);
      const float Sr = xh(iw) + q.wr;
      const float A2 = fmaf(Ar, Ar, q.wi2);
      const float S2 = fmaf(Sr, Sr, q.wi2);
      float r = rcp_approx_f32(A2 * S2);
      const float tr = fmaf(Kr, Ar, Kwr);
      const float ti = fmaf(Ki, Ar, Kwi);
      if (xrd > q.hi || xru < q.lo) {  // x outside the warp's interval
        branch1(iw, Ar, Sr, S2, r, tr, ti);
        continue;
      }
      float b2 = A2 * r;
      const float d = A2 - 0.25f;
      bool c1 = d > 0.0f;
      const bool near = fabsf(d) <= kMarginScale * (fabsf(xh(iw)) + kMarginW);
      const bool pole = A2 < kPoleA2;
      if (__any_sync(0xffffffffu, near || pole)) {
        if (near || pole) exact_decision<W>(*s_bt64, b * W + iw, sp, near, pole, c1, b2, r);
      }
      {  // inside the interval a warp is rarely all on branch 1: no vote, select per lane
        const unsigned m = smask(c1);
        const float a1 = msel(m, S2 * r, 0.0f);
        c[ci<W>(0, iw)] = fmaf(tr, a1, c[ci<W>(0, iw)]);
        c[ci<W>(1, iw)] = fmaf(ti, a1, c[ci<W>(1, iw)]);
        if (OCC) {
          // branch 2: M (-conj(S)/2) / |S|^2 = (Re M Yr - Im M Im w/2, Im M Yr + Re M Im w/2) b2
          // with Yr = -Sr/2
          const float wih = 0.5f * q.wi;
          const float coef = msel(m, r, b2);
          const float Yr = msel(m, fmaf(Ar, Sr, q.wi2), -0.5f * Sr);
          const float ur = fmaf(msel(m, K2r, Kr), Yr, msel(m, P1r, -Ki * wih));
          const float ui = fmaf(msel(m, K2i, Ki), Yr, msel(m, P1i, Kr * wih));
          c[ci<W>(2, iw)] = fmaf(ur, coef, c[ci<W>(2, iw)]);
          c[ci<W>(3, iw)] = fmaf(ui, coef, c[ci<W>(3, iw)]);
        }
      }
    }
  }
}

// All bands of one (igp, ig) pair: sum_b M F into the thread's band pairs (hi + lo, in
// shared memory, layout in F32Slots), which the caller multiplies by I w. Bands are summed
// in FP32 over chunks of kChunk bands and every chunk sum is added to the pair with Kahan's
// compensation. The FP64 wtilde is stored in the thread's slot for the exact path.
template <int W>
__device__ __forceinline__ void band_loop_f32(int B, int64_t G, int nocc,
                                              const float2* __restrict__ an_ptr,
                                              const float2* __restrict__ am_ptr,
                                              const float4* __restrict__ bt32,
                                              const BandEntry* const* s_bt64, double2 w64,
                                              bool live, float* sp) {
  PairF32 q;
  q.wr = static_cast<float>(w64.x);
  q.wr_lo = static_cast<float>(w64.x - static_cast<double>(q.wr));
  q.wi = static_cast<float>(w64.y);
  q.wi2 = q.wi * q.wi;
  q.w2i = 2.0f * q.wr * q.wi;           // Im w^2
  *F32Slots<W>::w64(sp) = w64;
#pragma unroll
  for (int k = 0; k < W; ++k) *F32Slots<W>::band4(sp, k) = make_float4(0.f, 0.f, 0.f, 0.f);
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
  // Kahan's summation over chunks: the running sums hi (shared memory) take each chunk sum,
  // and the rounding error of that addition, y - (t - hi), is carried in the chunk sums c
  // themselves (the next chunk's bands are added on top of it), so only hi is read and
  // written per merge; the last carry becomes the pairs' lo.
  float c[4 * W];
#pragma unroll
  for (int k = 0; k < 4 * W; ++k) c[k] = 0.0f;
#pragma unroll 1
  for (int b0 = 0; b0 < B; b0 += kChunk) {
    const int bend = min(b0 + kChunk, B);
    const int bocc = max(b0, min(nocc, bend));   // bands [b0, bocc) are occupied
    bands_f32<W, true>(b0, bocc, static_cast<int>(G), an_ptr, am_ptr, bt32, s_bt64, sp, q, c);
    if (bocc < bend)
      bands_f32<W, false>(bocc, bend, static_cast<int>(G), an_ptr, am_ptr, bt32, s_bt64, sp, q,
                          c);
#pragma unroll
    for (int qd = 0; qd < W; ++qd) {   // four values per shared-memory access
      float4 h = *F32Slots<W>::band4(sp, qd);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float& hi = quad_elem(h, i);
        float& y = c[ci<W>(i, qd)];
        const float t = hi + y;
        y = y - (t - hi);
        hi = t;
      }
      *F32Slots<W>::band4(sp, qd) = h;
    }
  }
#pragma unroll
  for (int qd = 0; qd < W; ++qd)
    *F32Slots<W>::band4(sp, W + qd) =
        make_float4(c[ci<W>(0, qd)], c[ci<W>(1, qd)], c[ci<W>(2, qd)], c[ci<W>(3, qd)]);
}

// (h, l) with h + l = a b exactly for FP32 a, b (no overflow or underflow): the product
// and its rounding error from a fused multiply-add.
__device__ __forceinline__ void two_prod(float a, float b, float& h, float& l) {
  h = a * b;
  l = fmaf(a, b, -h);
}

// Adds I w times the thread's band sums into its tile pairs (tp: 2W float4, hi quads then
// lo quads, in the thread's local memory), in double-FP32 arithmetic:
// with I w = (ar + ar_l) + i (ai + ai_l) (FP32 pairs of the FP64 product) and each band
// sum z = zh + zl, every real product is taken as its exact FP32 product plus the
// first-order cross terms, and added into the tile pair with pair_add. Relative error of
// order 2^-44 per value; FP32 operations only (the FP64 pipe is narrow). Band and tile
// quad iw hold the two complex values of frequency iw (Re ach, Im ach, Re asx, Im asx).
template <int W>
__device__ __noinline__ void fold_band_sums(float* sp, float4* tp, double2 Iw) {
  const float ar = static_cast<float>(Iw.x), ai = static_cast<float>(Iw.y);
  const float ar_l = static_cast<float>(Iw.x - static_cast<double>(ar));
  const float ai_l = static_cast<float>(Iw.y - static_cast<double>(ai));
#pragma unroll
  for (int qd = 0; qd < W; ++qd) {
    float4 zh = *F32Slots<W>::band4(sp, qd), zl = *F32Slots<W>::band4(sp, W + qd);
    float4 th = tp[qd], tl = tp[W + qd];
#pragma unroll
    for (int v = 0; v < 2; ++v) {  // complex value (components 2v: re, 2v + 1: im)
      const float zrh = quad_elem(zh, 2 * v), zrl = quad_elem(zl, 2 * v);
      const float zih = quad_elem(zh, 2 * v + 1), zil = quad_elem(zl, 2 * v + 1);
      // re = ar zr - ai zi,  im = ar zi + ai zr
      float p[4], e[4];
      two_prod(ar, zrh, p[0], e[0]);
      two_prod(ai, zih, p[1], e[1]);
      two_prod(ar, zih, p[2], e[2]);
      two_prod(ai, zrh, p[3], e[3]);
      e[0] = fmaf(ar, zrl, fmaf(ar_l, zrh, e[0]));
      e[1] = fmaf(ai, zil, fmaf(ai_l, zih, e[1]));
      e[2] = fmaf(ar, zil, fmaf(ar_l, zih, e[2]));
      e[3] = fmaf(ai, zrl, fmaf(ai_l, zrh, e[3]));
      pair_add(quad_elem(th, 2 * v), quad_elem(tl, 2 * v), p[0], e[0]);
      pair_add(quad_elem(th, 2 * v), quad_elem(tl, 2 * v), -p[1], -e[1]);
      pair_add(quad_elem(th, 2 * v + 1), quad_elem(tl, 2 * v + 1), p[2], e[2]);
      pair_add(quad_elem(th, 2 * v + 1), quad_elem(tl, 2 * v + 1), p[3], e[3]);
    }
    tp[qd] = th;
    tp[W + qd] = tl;
  }
}

}  // namespace gpp
