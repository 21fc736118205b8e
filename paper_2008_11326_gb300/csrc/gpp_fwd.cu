// Forward GPP sum in FP64: column gather, main sum, deterministic final reduction.
//
// Work decomposition (paper §III v4: the band loop runs serially inside a thread while
// (igp, ig) are spread over threads, which keeps every ig-contiguous array coalesced).
// A tile is one local column p and `threads` consecutive G-vectors; each thread owns one
// (p, ig) pair of the tile, hoists everything that depends on (p, ig) only, and walks all
// bands, evaluating every frequency iw from registers (the paper's v5 split of iw into
// separate launches would recompute the shared terms, which the narrow FP64 pipe of GB300
// cannot afford). The grid is persistent: CTA c takes tiles c, c + grid, ... in order, so
// the summation order, and therefore every bit of the result, is fixed.
//
// Arithmetic (paper §III v1: reciprocals instead of divides; §III v3: squared moduli).
// With A = x - w, S = x + w, C = x^2 - w^2 = A S, K = M I w, K2 = K w:
//   branch 1:  M sch = K / A        = K conj(A) / |A|^2
//              M ssx = M w^2 I / C  = K2 conj(C) / |C|^2
//   branch 2:  M ssx = -M I delw / (4 delw + 2) = -(K/2) / S = -(K/2) conj(S) / |S|^2
// (branch 2 uses delw = w / A, so 4 delw + 2 = 2 S / A). One reciprocal r = 1/(|A|^2 |S|^2)
// serves all three denominators: 1/|A|^2 = |S|^2 r, 1/|C|^2 = r, 1/|S|^2 = |A|^2 r.
// Branch selection picks operands (Z, Y, coefficient) for one shared complex
// multiply-accumulate, so a warp whose lanes take different branches pays once.

#include <cuda_runtime.h>

#include "gpp_device.cuh"
#include "gpp_internal.h"
#include "gpp_terms_f64.cuh"

namespace gpp {

namespace {


// Global column of local column p, or -1 if it contributes nothing. Counts indices that
// are outside their arrays (the sentinel indinv[k] == G is legitimate).
__device__ __forceinline__ int column_of(int64_t p, int64_t G, const int32_t* inv,
                                         const int32_t* indinv, int* bad) {
  int64_t k = inv[p];
  if (k < 0 || k > G) {
    if (bad) atomicAdd(bad, 1);
    return -1;
  }
  int64_t g = indinv[k];
  if (g < 0 || g > G) {
    if (bad) atomicAdd(bad, 1);
    return -1;
  }
  return g < G ? static_cast<int>(g) : -1;
}

// Column gather (paper §III v7: aqsmtemp_local(igp, band) stored band-contiguous),
// band tables and index checks. am32 / bt32 (the FP32-bulk copies) may be NULL.
__global__ void gpp_prep_kernel(int64_t B, int64_t G, int64_t P, int W,
                                const double2* __restrict__ aqsm,
                                const double* __restrict__ vcoul,
                                const int32_t* __restrict__ inv,
                                const int32_t* __restrict__ indinv,
                                const double* __restrict__ wx, int* flags, int* colg,
                                BandEntry* bt, double2* am, BandEntry32* bt32, float2* am32) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int64_t p = tid; p < P; p += stride) colg[p] = column_of(p, G, inv, indinv, flags + 1);
  for (int64_t i = tid; i < P * B; i += stride) {
    int64_t p = i / B, b = i - p * B;
    int g = column_of(p, G, inv, indinv, nullptr);
    double2 v = make_double2(0.0, 0.0);
    if (g >= 0) {
      double2 m = aqsm[b * G + g];
      double vc = vcoul[g];
      v = make_double2(m.x * vc, -m.y * vc);
    }
    am[i] = v;
    if (am32) am32[i] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
  }
  for (int64_t i = tid; i < B * W; i += stride) {
    double x = wx[i];
    bt[i] = BandEntry{make_double2(x, x * x), make_double2(4.0 * x, -0.5 * x)};
    if (!(x >= 0.0)) flags[0] = 1;
    if (!(fabs(x) < kFp32MaxX)) flags[2] = 1;
    if (bt32) {
      const float xf = static_cast<float>(x);
      BandEntry32 e;
      e.a = make_float4(xf, static_cast<float>(x * x), 4.0f * xf, -0.5f * xf);
      e.b = make_float4(kMarginScale * (fabsf(xf) + 2.0f), 0.0f, 0.0f, 0.0f);
      bt32[i] = e;
    }
  }
}

template <int W>
__global__ void __launch_bounds__(256) gpp_fwd_f64_kernel(
    int B, int64_t G, int nocc, int64_t n_ig_tiles, int64_t ntiles,
    const double2* __restrict__ aqsn, const double2* __restrict__ eps,
    const double2* __restrict__ wt, const double2* __restrict__ am,
    const BandEntry* __restrict__ bt, const int* __restrict__ colg,
    const int* __restrict__ flags, double* __restrict__ partials) {
  __shared__ double red[(256 / 32) * 4 * kMaxNw];
  double acc[4 * W];
#pragma unroll
  for (int k = 0; k < 4 * W; ++k) acc[k] = 0.0;
  const bool x_nonneg = flags[0] == 0;
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
    const double wr = w.x, wi = w.y;
    const double Iwr = fma(I.x, wr, -I.y * wi);
    const double Iwi = fma(I.x, wi, I.y * wr);
    const double wabs2 = fma(wr, wr, wi * wi);
    const bool fast_lane = wr >= 0.0 && gt_nonneg(wabs2, kFastWabs2Lo) &&
                           lt_nonneg(wabs2, kFastWabs2Hi);
    const double2* an_ptr = aqsn + (live ? ig : 0);
    const double2* am_ptr = am + p * B;
    if (__all_sync(0xffffffffu, fast_lane) && x_nonneg)
      band_loop<W, true>(B, G, nocc, an_ptr, am_ptr, bt, live, wr, wi, Iwr, Iwi, acc);
    else
      band_loop<W, false>(B, G, nocc, an_ptr, am_ptr, bt, live, wr, wi, Iwr, Iwi, acc);
  }
  block_partials<4 * W>(acc, red, partials + static_cast<int64_t>(blockIdx.x) * 4 * W);
}

// Fixed-order sum of the per-CTA partials: thread t adds partials t, t + 256, ... in order,
// then a pairwise tree over the 256 thread sums.
__global__ void __launch_bounds__(256) gpp_reduce_final_kernel(const double* __restrict__ part,
                                                               int nparts, int nv,
                                                               double* __restrict__ ach,
                                                               double* __restrict__ asx) {
  __shared__ double s[256];
  for (int k = 0; k < nv; ++k) {
    double v = 0.0;
    for (int j = threadIdx.x; j < nparts; j += 256) v += part[static_cast<int64_t>(j) * nv + k];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int iw = k / 4, c = k % 4;
      if (c < 2)
        ach[2 * iw + c] = s[0];
      else
        asx[2 * iw + c - 2] = s[0];
    }
    __syncthreads();
  }
}

template <int W>
cudaError_t launch_fwd_f64_w(const gpp_problem& p, int nocc, const FwdPlan& plan, char* ws,
                             cudaStream_t s) {
  gpp_fwd_f64_kernel<W><<<plan.grid, plan.threads, 0, s>>>(
      static_cast<int>(p.number_bands), p.ncouls, nocc, plan.n_ig_tiles, plan.ntiles,
      reinterpret_cast<const double2*>(p.aqsntemp),
      reinterpret_cast<const double2*>(p.I_eps_array),
      reinterpret_cast<const double2*>(p.wtilde_array),
      reinterpret_cast<const double2*>(ws + plan.off_am),
      reinterpret_cast<const BandEntry*>(ws + plan.off_bt),
      reinterpret_cast<const int*>(ws + plan.off_colvalid),
      reinterpret_cast<const int*>(ws + plan.off_flags),
      reinterpret_cast<double*>(ws + plan.off_partials));
  return cudaGetLastError();
}

template <int W>
const void* fwd_f64_fn() {
  return reinterpret_cast<const void*>(&gpp_fwd_f64_kernel<W>);
}

const void* fwd_f64_kernel_ptr(int nw) {
  switch (nw) {
    case 1: return fwd_f64_fn<1>();
    case 2: return fwd_f64_fn<2>();
    case 3: return fwd_f64_fn<3>();
    case 4: return fwd_f64_fn<4>();
    case 5: return fwd_f64_fn<5>();
    case 6: return fwd_f64_fn<6>();
    case 7: return fwd_f64_fn<7>();
    case 8: return fwd_f64_fn<8>();
    default: return nullptr;
  }
}

}  // namespace

int fwd_f64_blocks_per_sm(int threads, int nw) {
  const void* fn = fwd_f64_kernel_ptr(nw);
  if (!fn) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_prep(const gpp_problem& p, const FwdPlan& plan, char* ws, bool fp32,
                        cudaStream_t s) {
  int* flags = reinterpret_cast<int*>(ws + plan.off_flags);
  cudaError_t e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int64_t work = p.ngpown * p.number_bands + p.number_bands * p.nw + p.ngpown;
  int64_t blocks = (work + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  gpp_prep_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(
      p.number_bands, p.ncouls, p.ngpown, static_cast<int>(p.nw),
      reinterpret_cast<const double2*>(p.aqsmtemp), p.vcoul, p.inv_igp_index, p.indinv,
      p.wx_array, flags, reinterpret_cast<int*>(ws + plan.off_colvalid),
      reinterpret_cast<BandEntry*>(ws + plan.off_bt), reinterpret_cast<double2*>(ws + plan.off_am),
      fp32 ? reinterpret_cast<BandEntry32*>(ws + plan.off_bt32) : nullptr,
      fp32 ? reinterpret_cast<float2*>(ws + plan.off_am32) : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_fwd_f64(const gpp_problem& p, int occ_mode, const FwdPlan& plan, char* ws,
                           cudaStream_t s) {
  int64_t nocc = p.number_bands;
  if (occ_mode == GPP_OCC_OCCUPIED) nocc = p.nvband < p.number_bands ? p.nvband : p.number_bands;
  const int n = static_cast<int>(nocc);
  switch (p.nw) {
    case 1: return launch_fwd_f64_w<1>(p, n, plan, ws, s);
    case 2: return launch_fwd_f64_w<2>(p, n, plan, ws, s);
    case 3: return launch_fwd_f64_w<3>(p, n, plan, ws, s);
    case 4: return launch_fwd_f64_w<4>(p, n, plan, ws, s);
    case 5: return launch_fwd_f64_w<5>(p, n, plan, ws, s);
    case 6: return launch_fwd_f64_w<6>(p, n, plan, ws, s);
    case 7: return launch_fwd_f64_w<7>(p, n, plan, ws, s);
    case 8: return launch_fwd_f64_w<8>(p, n, plan, ws, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_reduce_final(const FwdPlan& plan, char* ws, gpp_c128* ach, gpp_c128* asx,
                                cudaStream_t s) {
  gpp_reduce_final_kernel<<<1, 256, 0, s>>>(reinterpret_cast<const double*>(ws + plan.off_partials),
                                            plan.grid, 4 * plan.nw,
                                            reinterpret_cast<double*>(ach),
                                            reinterpret_cast<double*>(asx));
  return cudaGetLastError();
}

}  // namespace gpp
