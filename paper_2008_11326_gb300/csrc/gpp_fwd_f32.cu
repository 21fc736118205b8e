// Forward GPP sum with FP32 bulk arithmetic (GPP_FP32_BULK).
//
// Same decomposition and algebra as the FP64 kernel (gpp_fwd.cu), with the per-term
// complex arithmetic in FP32 on complex64 data: the band-indexed aqsntemp is read from
// its complex64 copy and the gathered weights conj(aqsmtemp) vcoul are rounded once by
// the gather kernel; wtilde and I_eps are read in FP64 once per (igp, ig) pair and rounded
// in registers. FP64 is kept where FP32 would change the answer:
//
//  * Branch decisions. The branch taken at |wdiff|^2 = 1/4 is discontinuous, and FP32
//    rounding of x and w moves |wdiff|^2 by ~1e-7: on the benchmark shape thousands of
//    terms would switch branch, an error of order 1e-4 in the sums. The kernel therefore
//    evaluates d = |wdiff|^2 - 1/4 in FP32 together with a bound m on its rounding error,
//        m = 2^-20 (|x| + |Re w| + 2),
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

#include <cuda_runtime.h>

#include "gpp_device.cuh"
#include "gpp_internal.h"
#include "gpp_terms_f32.cuh"
#include "gpp_terms_f64.cuh"

namespace gpp {

namespace {

template <int W>
__global__ void __launch_bounds__(256) gpp_fwd_f32_kernel(
    int B, int64_t G, int nocc, int64_t n_ig_tiles, int64_t ntiles,
    const double2* __restrict__ aqsn64, const float2* __restrict__ aqsn32,
    const double2* __restrict__ eps, const double2* __restrict__ wt,
    const double2* __restrict__ am64, const float2* __restrict__ am32,
    const BandEntry* __restrict__ bt64, const BandEntry32* __restrict__ bt32,
    const int* __restrict__ colg, const int* __restrict__ flags, double* __restrict__ partials) {
  __shared__ double red[(256 / 32) * 4 * kMaxNw];
  double acc[4 * W];
#pragma unroll
  for (int k = 0; k < 4 * W; ++k) acc[k] = 0.0;
  const bool x_fast = flags[0] == 0 && flags[2] == 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p = t / n_ig_tiles;
    const int64_t ig = (t - p * n_ig_tiles) * blockDim.x + threadIdx.x;
    const bool live = ig < G && colg[p] >= 0;
    double2 w = make_double2(0.5, 1.0);  // inert lane: finite terms, zero weight
    double2 I = make_double2(0.0, 0.0);
    if (live) {
      w = ldg2(wt + p * G + ig);
      I = ldg2(eps + p * G + ig);
    }
    const double wabs2 = fma(w.x, w.x, w.y * w.y);
    const bool fast_lane = w.x >= 0.0 && gt_nonneg(wabs2, kFastWabs2Lo) &&
                           lt_nonneg(wabs2, kFastWabs2Hi);
    if (__all_sync(0xffffffffu, fast_lane) && x_fast) {
      band_loop_f32<W>(B, G, nocc, aqsn32 + (live ? ig : 0), am32 + p * B, bt32, bt64, w, I, acc);
    } else {
      const double Iwr = fma(I.x, w.x, -I.y * w.y);
      const double Iwi = fma(I.x, w.y, I.y * w.x);
      band_loop<W, false>(B, G, nocc, aqsn64 + (live ? ig : 0), am64 + p * B, bt64, live, w.x,
                          w.y, Iwr, Iwi, acc);
    }
  }
  block_partials<4 * W>(acc, red, partials + static_cast<int64_t>(blockIdx.x) * 4 * W);
}

template <int W>
cudaError_t launch_w(const gpp_problem& p, int nocc, const FwdPlan& plan, char* ws,
                     cudaStream_t s) {
  gpp_fwd_f32_kernel<W><<<plan.grid, plan.threads, 0, s>>>(
      static_cast<int>(p.number_bands), p.ncouls, nocc, plan.n_ig_tiles, plan.ntiles,
      reinterpret_cast<const double2*>(p.aqsntemp),
      reinterpret_cast<const float2*>(p.aqsntemp_c64),
      reinterpret_cast<const double2*>(p.I_eps_array),
      reinterpret_cast<const double2*>(p.wtilde_array),
      reinterpret_cast<const double2*>(ws + plan.off_am),
      reinterpret_cast<const float2*>(ws + plan.off_am32),
      reinterpret_cast<const BandEntry*>(ws + plan.off_bt),
      reinterpret_cast<const BandEntry32*>(ws + plan.off_bt32),
      reinterpret_cast<const int*>(ws + plan.off_colvalid),
      reinterpret_cast<const int*>(ws + plan.off_flags),
      reinterpret_cast<double*>(ws + plan.off_partials));
  return cudaGetLastError();
}

template <int W>
const void* kernel_fn() {
  return reinterpret_cast<const void*>(&gpp_fwd_f32_kernel<W>);
}

const void* kernel_ptr(int nw) {
  switch (nw) {
    case 1: return kernel_fn<1>();
    case 2: return kernel_fn<2>();
    case 3: return kernel_fn<3>();
    case 4: return kernel_fn<4>();
    case 5: return kernel_fn<5>();
    case 6: return kernel_fn<6>();
    case 7: return kernel_fn<7>();
    case 8: return kernel_fn<8>();
    default: return nullptr;
  }
}

}  // namespace

bool fwd_f32_available() { return true; }

int fwd_f32_blocks_per_sm(int threads, int nw) {
  const void* fn = kernel_ptr(nw);
  if (!fn) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_fwd_f32(const gpp_problem& p, int occ_mode, const FwdPlan& plan, char* ws,
                           cudaStream_t s) {
  int64_t nocc = p.number_bands;
  if (occ_mode == GPP_OCC_OCCUPIED) nocc = p.nvband < p.number_bands ? p.nvband : p.number_bands;
  const int n = static_cast<int>(nocc);
  switch (p.nw) {
    case 1: return launch_w<1>(p, n, plan, ws, s);
    case 2: return launch_w<2>(p, n, plan, ws, s);
    case 3: return launch_w<3>(p, n, plan, ws, s);
    case 4: return launch_w<4>(p, n, plan, ws, s);
    case 5: return launch_w<5>(p, n, plan, ws, s);
    case 6: return launch_w<6>(p, n, plan, ws, s);
    case 7: return launch_w<7>(p, n, plan, ws, s);
    case 8: return launch_w<8>(p, n, plan, ws, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gpp
