// Device-side building blocks shared by the GPP kernels: constants of the plasmon-pole
// branch, the FP64 reciprocal, bit-pattern comparisons and the deterministic reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpp {

// Thresholds of the three-way branch (paper §III v2), compared against squared moduli
// (§III v3): |wdiff|^2 > LIMITTWO and |delw|^2 < LIMITONE select branch 1, otherwise
// |delw|^2 > TOL_ZERO selects branch 2.
constexpr double kLimitTwo = 0.25;
constexpr double kLimitOne = 250000.0;  // 1 / (4 * 1e-6)
constexpr double kTolZero = 1.0e-12;
constexpr long long kLimitTwoBits = 0x3FD0000000000000LL;  // bit pattern of 0.25

// The fast path decides branch 1 from |wdiff|^2 alone. That is exact when
// 1e-12 < |w|^2 < 62499: then |wdiff|^2 > 1/4 implies |delw|^2 = |w|^2/|wdiff|^2 < 249996
// (below LIMITONE by far more than rounding), and |wdiff|^2 <= 1/4 implies
// |delw|^2 >= 4|w|^2 > TOL_ZERO.
constexpr double kFastWabs2Lo = 1.0e-12;
constexpr double kFastWabs2Hi = 62499.0;

constexpr int kMaxNw = 8;

// One (band, iw) entry of the FP64 band table: x = wx_array[b][iw], x^2 and -x/2 (hi.x pads
// the entry to 32 bytes).
struct alignas(32) BandEntry {
  double2 lo;  // x, x^2
  double2 hi;  // 0, -x/2
};

// The FP32 band table: per band, f32_band_quads(W) float4: x_hi[0..W-1] (each frequency
// rounded to FP32) then the minimum of the band's frequencies rounded down, padded to whole
// float4; then x_lo[0..W-1] (the FP32 residuals x - x_hi) and the maximum rounded up,
// likewise (two float4, 32 bytes, for W <= 3). The per-lane path derives its bounds on x
// and its decision margin from x_hi (gpp_terms_f32.cuh).
__host__ __device__ constexpr int f32_half_quads(int W) { return (W + 4) / 4; }
__host__ __device__ constexpr int f32_band_quads(int W) { return 2 * f32_half_quads(W); }

// Flags written by the gather kernel: [0] some wx < 0 or NaN, [1] bad index count,
// [2] some |wx| >= kFp32MaxX or NaN (the FP32 decision margin assumes smaller x); from int
// kFlagXmax on, the bits of max |wx| as a 64-bit integer. kFlagBytes in all.
constexpr double kFp32MaxX = 1.0e4;
constexpr int kFlagXmax = 4;
constexpr size_t kFlagBytes = 4 * sizeof(int) + sizeof(unsigned long long);

// The FP64 fast paths (forward and adjoint) take the asxtemp terms in partial fractions,
// M w / (A S) = (M/A - M/S) / 2, whose subtraction loses about log2(1 + x / |w|) bits where
// the two parts nearly cancel (x >> |w|). A warp takes them only if every lane has
// |w| >= max|wx| / 128 (|w|^2 >= kPfRatio2 max|wx|^2), which bounds the loss to 7 bits
// (relative errors of a few 1e-14 instead of a few 1e-16); other warps take the general
// form, which does not cancel.
constexpr double kPfRatio2 = 1.0 / 16384.0;

// The smallest |w|^2 of a warp on the partial-fraction fast path, from the gather's flags.
__device__ __forceinline__ double pf_wabs2_min(const int* flags) {
  const double xmax = __longlong_as_double(
      static_cast<long long>(*reinterpret_cast<const unsigned long long*>(flags + kFlagXmax)));
  return kPfRatio2 * xmax * xmax;
}

// The FP32 branch-decision margin 2^-20 (|x| + kMarginW) (see gpp_terms_f32.cuh); kMarginW
// bounds |Re w| + 2 on the fast path, where |w|^2 < kFastWabs2Hi.
constexpr float kMarginScale = 9.5367431640625e-07f;
constexpr float kMarginW = 252.0f;

// Ordering of non-negative doubles equals the ordering of their bit patterns as signed
// 64-bit integers. The comparisons below run on the integer pipe instead of the FP64 pipe
// (on GB300 the FP64 pipe is the bottleneck of the whole sum). Arguments are >= +0 or NaN.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ bool gt_nonneg(double a, double b) { return dbits(a) > dbits(b); }
__device__ __forceinline__ bool lt_nonneg(double a, double b) { return dbits(a) < dbits(b); }

// x / 2 on the integer pipe (the FP64 pipe is the FP64 kernel's bottleneck): one off the
// exponent field. Exact when that field is in [2, 2046]; +-0, subnormal and smallest-normal
// x give a signed zero (an absolute error below 2^-1022); infinities and NaN pass through.
__device__ __forceinline__ double half_alu(double x) {
  const long long b = __double_as_longlong(x);
  const int e = static_cast<int>((b >> 52) & 0x7ff);
  long long h = (e >= 2) ? b - (1LL << 52) : (b & (1LL << 63));
  h = (e == 0x7ff) ? b : h;
  return __longlong_as_double(h);
}

// 2 x on the integer pipe: one onto the exponent field. Exact for finite x below the
// largest binade; a subnormal or zero x has its bits shifted left (also exact), a result
// past the largest finite double becomes an infinity, infinities and NaN pass through.
__device__ __forceinline__ double twice_alu(double x) {
  const long long b = __double_as_longlong(x);
  const long long sign = b & (1LL << 63);
  const int e = static_cast<int>((b >> 52) & 0x7ff);
  long long h = b + (1LL << 52);
  h = (e == 0) ? (sign | ((b & ~(1LL << 63)) << 1)) : h;
  h = (e == 0x7fe) ? (sign | 0x7ff0000000000000LL) : h;
  h = (e == 0x7ff) ? b : h;
  return __longlong_as_double(h);
}

// FP64 reciprocal: the hardware approximation (PTX rcp.approx.ftz.f64) refined by one
// third-order Householder step of Newton's reciprocal iteration,
//   e = 1 - d*y,   y' = y * (1 + e + e^2),
// whose relative error is e^3 plus rounding. Three FP64 FMAs instead of the longer
// correctly-rounded sequence; the result differs from 1/d by a few ulp at most (checked
// against 1.0/d by the test suite). d must be a normal, finite, non-zero double.
__device__ __forceinline__ double rcp_approx(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  return y;
}

__device__ __forceinline__ double rcp_refined(double d) {
  double y = rcp_approx(d);
  double e = fma(-d, y, 1.0);
  double q = fma(e, e, e);
  return fma(y, q, y);
}

__device__ __forceinline__ double2 ldg2(const double2* p) { return __ldg(p); }

// Sum of v over the warp by a fixed xor butterfly; lane 0's result is deterministic.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Per-CTA partial of NV doubles: warp butterflies, then warp partials summed in warp
// order by the first NV threads. `red` is shared memory of at least (blockDim/32) * NV.
template <int NV>
__device__ __forceinline__ void block_partials(double (&acc)[NV], double* red, double* out) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double v = warp_sum(acc[k]);
    if (lane == 0) red[warp * NV + k] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += red[w * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// Compensated FP32 pair arithmetic (hi + lo, |lo| << |hi|): (hi, lo) += (bh, bl) with
// Knuth's TwoSum on the leading parts, so the pair carries about twice FP32's precision.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float v = s - hi;
  const float e = (hi - (s - v)) + (bh - v);
  lo = lo + bl + e;
  hi = s;
}

// Per-CTA partial of NV compensated FP32 pairs: warp butterflies and a warp-order sum, all
// with pair_add; `red` is shared memory of at least (blockDim/32) * NV float2.
template <int NV>
__device__ __forceinline__ void block_pairs(float (&hi)[NV], float (&lo)[NV], float2* red,
                                            float2* out) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float h = hi[k], l = lo[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, off);
      const float ol = __shfl_xor_sync(0xffffffffu, l, off);
      pair_add(h, l, oh, ol);
    }
    if (lane == 0) red[warp * NV + k] = make_float2(h, l);
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    float h = 0.0f, l = 0.0f;
    for (int w = 0; w < nwarps; ++w) {
      const float2 v = red[w * NV + threadIdx.x];
      pair_add(h, l, v.x, v.y);
    }
    out[threadIdx.x] = make_float2(h, l);
  }
}

}  // namespace gpp
