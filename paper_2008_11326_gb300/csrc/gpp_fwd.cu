// Forward GPP sum: the column gather. The main sum runs in gpp_batched.cu (a single
// instance is a batch of one) with the per-band arithmetic of gpp_terms_f64.cuh and
// gpp_terms_f32.cuh.
//
// Work decomposition (paper §III v4: the band loop runs serially inside a thread while
// (igp, ig) are spread over threads, which keeps every ig-contiguous array coalesced).
// A tile is one local column p and `threads * ig_per_thread` consecutive G-vectors; each
// thread owns (p, ig) pairs of the tile, hoists everything that depends on (p, ig) only,
// and walks all bands, evaluating every frequency iw from registers (the paper's v5 split
// of iw into separate launches would recompute the shared terms, which the narrow FP64
// pipe of GB300 cannot afford). Every tile writes its own partial and the partials are
// summed in tile order, so every bit of the result is fixed.
//
// Arithmetic (paper §III v1: reciprocals instead of divides; §III v3: squared moduli).
// With A = x - w, S = x + w, C = x^2 - w^2 = A S, K = M I w, K2 = K w:
//   branch 1:  M sch = K / A        = K conj(A) / |A|^2
//              M ssx = M w^2 I / C  = K2 conj(C) / |C|^2 = (K/A - K/S) / 2
//   branch 2:  M ssx = -M I delw / (4 delw + 2) = -(K/2) / S = -(K/2) conj(S) / |S|^2
// (branch 2 uses delw = w / A, so 4 delw + 2 = 2 S / A; branch 1's partial fractions use
// S - A = 2 w). On the fast path, where branch 3 cannot occur, asxtemp is therefore
// (achtemp - sum K/S) / 2 over the occupied bands: two reciprocals per term, 1/|A|^2 and
// 1/|S|^2, and no branch on the asxtemp side. The general form (both thresholds and the
// screened-exchange cutoff) keeps one reciprocal r = 1/(|A|^2 |S|^2) for all three
// denominators, 1/|A|^2 = |S|^2 r, 1/|C|^2 = r, 1/|S|^2 = |A|^2 r, and branch selection picks
// operands (Z, Y, coefficient) for one shared complex multiply-accumulate, so a warp whose
// lanes take different branches pays once.

#include <cuda_runtime.h>

#include <algorithm>

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
// band tables and index checks. am32 / bt32 (the FP32-bulk copies) may be NULL. For a
// single-instance call the kernel also writes the instance descriptor the main kernel
// reads (so the call needs no host-to-device copy and can be captured in a graph).
__global__ void gpp_prep_kernel(int64_t B, int64_t G, int64_t P, int W,
                                const double2* __restrict__ aqsm,
                                const double* __restrict__ vcoul,
                                const int32_t* __restrict__ inv,
                                const int32_t* __restrict__ indinv,
                                const double* __restrict__ wx, int* flags, int* colg,
                                BandEntry* bt, double2* am, float4* bt32, float2* am32,
                                BatchInst* desc_out, const BatchInst desc) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (desc_out && tid == 0) *desc_out = desc;
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
    bt[i] = BandEntry{make_double2(x, x * x), make_double2(0.0, -0.5 * x)};
    if (!(x >= 0.0)) flags[0] = 1;
    if (!(fabs(x) < kFp32MaxX)) flags[2] = 1;
    // max |wx|: non-negative doubles order as their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(flags + kFlagXmax),
              static_cast<unsigned long long>(__double_as_longlong(fabs(x))));
    if (bt32) {  // layout of f32_band_quads (gpp_device.cuh)
      const float xf = static_cast<float>(x);
      const int64_t b0 = i / W, iw = i - b0 * W;
      const int nq = (W + 4) / 4;
      float* fb = reinterpret_cast<float*>(bt32 + b0 * (2 * nq));
      fb[iw] = xf;
      fb[4 * nq + iw] = static_cast<float>(x - static_cast<double>(xf));
      if (iw == 0) {  // the band's frequency range, rounded outwards, and the padding
        float lo = __int_as_float(0x7f800000), hi = -lo;
        for (int k = 0; k < W; ++k) {
          lo = fminf(lo, __double2float_rd(wx[b0 * W + k]));
          hi = fmaxf(hi, __double2float_ru(wx[b0 * W + k]));
        }
        fb[W] = lo;
        fb[4 * nq + W] = hi;
        for (int k = W + 1; k < 4 * nq; ++k) fb[k] = fb[4 * nq + k] = 0.0f;
      }
    }
  }
}

// Complex128 -> complex64 (round to nearest) over a block of rows x columns: the FP32-bulk
// copy of aqsntemp when the caller passes none. A streaming copy (read 16 bytes, write 8 per
// element), bound by HBM.
__global__ void gpp_convert_c64_kernel(const double2* __restrict__ src, int64_t ld_src,
                                       float2* __restrict__ dst, int64_t ld_dst, int64_t rows,
                                       int64_t c0, int64_t ncols) {
  const int64_t n = rows * ncols;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += stride) {
    const int64_t r = i / ncols, c = c0 + (i - r * ncols);
    const double2 v = __ldcs(src + r * ld_src + c);
    __stcs(dst + r * ld_dst + c, make_float2(static_cast<float>(v.x), static_cast<float>(v.y)));
  }
}

}  // namespace

cudaError_t launch_convert_c64(const gpp_c128* src, int64_t ld_src, gpp_c64* dst, int64_t ld_dst,
                               int64_t rows, int64_t c0, int64_t c1, cudaStream_t s) {
  const int64_t n = rows * (c1 - c0);
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // a grid of whole waves (8 CTAs of 256 threads per SM), fewer for small copies
  int64_t blocks = std::min<int64_t>((n + 255) / 256, static_cast<int64_t>(sms) * 8);
  gpp_convert_c64_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(
      reinterpret_cast<const double2*>(src), ld_src, reinterpret_cast<float2*>(dst), ld_dst,
      rows, c0, c1 - c0);
  return cudaGetLastError();
}

cudaError_t launch_prep(const gpp_problem& p, const FwdPlan& plan, char* ws, bool fp32,
                        const BatchInst* desc, cudaStream_t s) {
  int* flags = reinterpret_cast<int*>(ws + plan.off_flags);
  cudaError_t e = cudaMemsetAsync(flags, 0, kFlagBytes, s);
  if (e != cudaSuccess) return e;
  if (fp32 && plan.convert_c64) {
    e = launch_convert_c64(p.aqsntemp, p.ncouls, reinterpret_cast<gpp_c64*>(ws + plan.off_aqsn32),
                           p.ncouls, p.number_bands, 0, p.ncouls, s);
    if (e != cudaSuccess) return e;
  }
  const int64_t work = p.ngpown * p.number_bands + p.number_bands * p.nw + p.ngpown;
  int64_t blocks = (work + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  gpp_prep_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(
      p.number_bands, p.ncouls, p.ngpown, static_cast<int>(p.nw),
      reinterpret_cast<const double2*>(p.aqsmtemp), p.vcoul, p.inv_igp_index, p.indinv,
      p.wx_array, flags, reinterpret_cast<int*>(ws + plan.off_colvalid),
      reinterpret_cast<BandEntry*>(ws + plan.off_bt), reinterpret_cast<double2*>(ws + plan.off_am),
      fp32 ? reinterpret_cast<float4*>(ws + plan.off_bt32) : nullptr,
      fp32 ? reinterpret_cast<float2*>(ws + plan.off_am32) : nullptr,
      desc ? reinterpret_cast<BatchInst*>(ws + plan.off_desc) : nullptr, desc ? *desc : BatchInst());
  return cudaGetLastError();
}

}  // namespace gpp
