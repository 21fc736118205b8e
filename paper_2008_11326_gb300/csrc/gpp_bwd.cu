// Adjoint of the GPP sum in FP64 (gpp_sigma_backward).
//
// The loss seen by the adjoint is L with dL = Re(sum_iw conj(g_ach[iw]) d achtemp[iw] +
// conj(g_asx[iw]) d asxtemp[iw]) (PyTorch's convention for complex outputs). With
// c_a = conj(g_ach), c_s = conj(g_asx) and the per-term weight M = am * aqsntemp (am =
// conj(aqsmtemp[b][g]) vcoul[g]), every (b, p, ig) contributes M Q to L, where
//   Q   = I w GI,   GI = sum_iw  c_a [b1] u  +  c_s occ (b1 ? w u v : -v/2)
//   dQ/dw-part:     GW = sum_iw  c_a [b1] x u^2  +  c_s occ (b1 ? 2 x^2 w (u v)^2 : -x v^2 / 2)
// with u = 1/(x - w), v = 1/(x + w) (so w u = delw, w^2 u v = w^2/(x^2 - w^2)); these are the
// derivatives of the branch formulas (the branch predicates are locally constant). Then
//   grad wtilde[p][ig]   = conj( sum_b M I GW )         (holomorphic input)
//   grad I_eps[p][ig]    = conj( sum_b M w GI )
//   grad aqsntemp[b][ig] = conj( sum_p am Q )
//   grad aqsmtemp[b][g]  = vcoul[g] sum_{p: g(p) = g} sum_ig aqsntemp[b][ig] Q   (enters
//                          through its conjugate, so no outer conj)
// Terms are recomputed, not stored. One reciprocal r = 1/(|x-w|^2 |x+w|^2) per term gives
// u = conj(x-w)|x+w|^2 r, v = conj(x+w)|x-w|^2 r and u v = conj(x^2-w^2) r.
//
// Decomposition: a CTA owns a tile of 8 columns (threadIdx.y) x 32 G-vectors (threadIdx.x),
// one (p, ig) pair per thread, and walks every band. wtilde / I_eps gradients stay in
// registers. Per band, the CTA reduces am Q over its 8 columns and aqsntemp Q over its 32
// G-vectors in shared memory with a fixed tree and writes one partial per tile; columns are
// processed in batches of kBatchGroups column groups per launch, and a finishing kernel
// adds each batch's partials into the outputs in a fixed order. No atomics: results are
// deterministic.

#include <cuda_runtime.h>

#include "gpp_device.cuh"
#include "gpp_internal.h"

namespace gpp {

namespace {

constexpr int kTX = 32;  // G-vectors per tile
constexpr int kTY = 8;   // columns per tile (one column group)

// One (band, iw) entry for the adjoint: x, x^2 and the cotangent products that do not
// depend on (p, ig): c_a + c_s / 2 and its product with x (the fast path's partial
// fractions), c_a, c_s, c_a x, -c_s / 2, -x c_s / 2.
struct alignas(32) BwdBand {
  double2 lo;     // x, x^2
  double2 cap;    // c_a + c_s / 2
  double2 ca;     // c_a
  double2 cs;     // c_s
  double2 cax;    // c_a x
  double2 capx;   // (c_a + c_s / 2) x
  double2 csh;    // -c_s / 2
  double2 csxh;   // -x c_s / 2
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__device__ __forceinline__ double2 csel(bool c, double2 a, double2 b) { return c ? a : b; }

template <bool V>
struct BoolTag {
  static constexpr bool value = V;
};

// ach_scale: 1/2 with the half Coulomb-hole factor (it scales every achtemp cotangent).
__global__ void gpp_bwd_prep_kernel(int64_t B, int W, const double* __restrict__ wx,
                                    const double2* __restrict__ g_ach,
                                    const double2* __restrict__ g_asx, double ach_scale,
                                    BwdBand* bt) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < B * W;
       i += stride) {
    const int iw = static_cast<int>(i % W);
    const double x = wx[i];
    const double2 ga = g_ach[iw], gs = g_asx[iw];
    const double2 ca = make_double2(ach_scale * ga.x, -ach_scale * ga.y);
    const double2 cs = make_double2(gs.x, -gs.y);
    BwdBand e;
    e.lo = make_double2(x, x * x);
    e.cap = make_double2(ca.x + 0.5 * cs.x, ca.y + 0.5 * cs.y);
    e.ca = ca;
    e.cs = cs;
    e.cax = make_double2(ca.x * x, ca.y * x);
    e.capx = make_double2(e.cap.x * x, e.cap.y * x);
    e.csh = make_double2(-0.5 * cs.x, -0.5 * cs.y);
    e.csxh = make_double2(-0.5 * x * cs.x, -0.5 * x * cs.y);
    bt[i] = e;
  }
}

// z^2 for a complex z, with the doubling of the imaginary part on the integer pipe.
__device__ __forceinline__ double2 csq(double2 z) {
  return make_double2(fma(z.x, z.x, -z.y * z.y), twice_alu(z.x * z.y));
}

// Per-term work for one band, all frequencies, on the fast path (every lane of the warp has
// 1e-12 < |w|^2 < 62499 and Re w >= 0, every wx >= 0: branch 1 is exactly |x - w|^2 > 1/4,
// branch 3 and the screened-exchange cutoff cannot occur). In partial fractions, with
// u = 1/(x - w), v = 1/(x + w) and b1 the branch-1 predicate, the asxtemp parts are
// w u v = (u - v)/2 and -v/2 in GI, 2 x^2 w (u v)^2 = x (u^2 - v^2)/2 and -x v^2/2 in GW, so
//   GI = sum_iw (c_a + c_s/2) b1 u - (c_s/2) v,   GW = sum_iw (c_a + c_s/2) b1 x u^2 - (c_s/2) x v^2
// on occupied bands (c_a b1 u and c_a b1 x u^2 on the others): two reciprocals per term and
// a select on u only.
template <int W, bool OCC>
__device__ __forceinline__ void bwd_terms_fast(const BwdBand* __restrict__ e, double wr,
                                               double wi, double wi2, double2& GI,
                                               double2& GW) {
#pragma unroll
  for (int iw = 0; iw < W; ++iw) {
    const double x = __ldg(&e[iw].lo.x);
    const double Ar = x - wr;
    const double A2 = fma(Ar, Ar, wi2);
    const double ra = rcp_refined(A2);
    const bool c1 = gt_nonneg(A2, kLimitTwo);
    const double2 u = c1 ? make_double2(Ar * ra, wi * ra) : make_double2(0.0, 0.0);
    const double2 uu = csq(u);
    if (OCC) {
      const double Sr = x + wr;
      const double S2 = fma(Sr, Sr, wi2);        // >= |w|^2 > 1e-12
      const double rs = rcp_refined(S2);
      const double2 v = make_double2(Sr * rs, -wi * rs);
      cmac(GI, __ldg(&e[iw].cap), u);
      cmac(GI, __ldg(&e[iw].csh), v);
      cmac(GW, __ldg(&e[iw].capx), uu);
      cmac(GW, __ldg(&e[iw].csxh), csq(v));
    } else {
      cmac(GI, __ldg(&e[iw].ca), u);
      cmac(GW, __ldg(&e[iw].cax), uu);
    }
  }
}

// Per-term work for one band, all frequencies, in the general form: accumulates GI and GW.
// sx2: sexcut^2 of the screened-exchange cutoff, 0 = off; where it drops ssx (x < 0 and
// |ssx| / |I| > sexcut, tested as in the forward) the ssx derivatives are zero.
template <int W, bool OCC>
__device__ __forceinline__ void bwd_terms(const BwdBand* __restrict__ e, double wr,
                                          double wi, double wi2, double wabs2, double mw2r,
                                          double w2i, double2 w, double sx2, double2& GI,
                                          double2& GW) {
#pragma unroll
  for (int iw = 0; iw < W; ++iw) {
    const double2 lo = __ldg(&e[iw].lo);
    const double x = lo.x, x2 = lo.y;
    const double Ar = x - wr;
    const double A2 = fma(Ar, Ar, wi2);
    const double Sr = x + wr;
    const double S2 = fma(Sr, Sr, wi2);
    const bool c1 = gt_nonneg(A2, kLimitTwo) && lt_nonneg(wabs2, kLimitOne * A2);
    const bool c2 = gt_nonneg(wabs2, kTolZero * A2);
    const double r = rcp_refined(A2 * S2);
    const double a1 = c1 ? S2 * r : 0.0;
    const double2 u = make_double2(Ar * a1, wi * a1);          // 1/(x - w) on branch 1
    cmac(GI, __ldg(&e[iw].ca), u);
    cmac(GW, __ldg(&e[iw].cax), cmul(u, u));
    if (OCC) {
      const double b2 = A2 * r;
      const double2 v = make_double2(Sr * b2, -wi * b2);       // 1/(x + w)
      const double2 uv = make_double2((x2 + mw2r) * r, w2i * r);  // 1/(x^2 - w^2)
      const double2 wuv = cmul(w, uv);
      const double2 h = csel(c1, wuv, v);
      const double2 T = cmul(h, csel(c1, uv, v));   // w (uv)^2 or v^2
      const double2 zero = make_double2(0.0, 0.0);
      const bool keep = !(sx2 > 0.0 && x < 0.0 &&
                          (c1 ? gt_nonneg(wabs2 * wabs2 * r, sx2)
                              : gt_nonneg(wabs2, 4.0 * sx2 * S2)));
      const double2 cs = __ldg(&e[iw].cs);
      const double tx2 = 2.0 * x2;
      const double2 cs2x2 = make_double2(tx2 * cs.x, tx2 * cs.y);   // 2 x^2 c_s
      const double2 ch = !keep ? zero : c1 ? cs : (c2 ? __ldg(&e[iw].csh) : zero);
      const double2 cT = !keep ? zero : c1 ? cs2x2 : (c2 ? __ldg(&e[iw].csxh) : zero);
      cmac(GI, ch, h);
      cmac(GW, cT, T);
    }
  }
}

// Fixed shared-memory trees: sums s_a[ty][tx] over ty (into s_a[0][tx]) and s_r[ty][tx]
// over tx (into s_r[ty][0]). The 256 threads are numbered L = 32 ty + tx and each level's
// additions go to the lowest L, so every level but the last two of the row tree runs on
// whole warps (a partly masked warp costs the FP64 pipe as much as a full one): 32 warp
// additions per band instead of 94 with one row per warp. The two trees share the
// barriers.
__device__ __forceinline__ void tile_reduce(double2 (*s_a)[kTX], double2 (*s_r)[kTX]) {
  const int L = threadIdx.y * kTX + threadIdx.x;
#pragma unroll
  for (int lev = 0; lev < 5; ++lev) {
    const int hr = (kTX / 2) >> lev;           // row tree: 16, 8, 4, 2, 1
    if (L < kTY * hr) {
      const int row = L / hr, col = L - row * hr;
      s_r[row][col].x += s_r[row][col + hr].x;
      s_r[row][col].y += s_r[row][col + hr].y;
    }
    if (lev < 3) {
      const int hc = (kTY / 2) >> lev;         // column tree: 4, 2, 1
      if (L < kTX * hc) {
        const int row = L / kTX, col = L - row * kTX;
        s_a[row][col].x += s_a[row + hc][col].x;
        s_a[row][col].y += s_a[row + hc][col].y;
      }
    }
    __syncthreads();
  }
}

template <int W>
__global__ void __launch_bounds__(kTX * kTY, 2) gpp_bwd_kernel(
    int B, int64_t G, int64_t P, int nocc, int64_t group0, int ngroups, int64_t n_ig_tiles,
    const double2* __restrict__ aqsn, const double2* __restrict__ eps,
    const double2* __restrict__ wt, const double2* __restrict__ am,
    const BwdBand* __restrict__ bt, const int* __restrict__ colg, const int* __restrict__ flags,
    double2* __restrict__ grad_w, double2* __restrict__ grad_I,
    double2* __restrict__ part_n,  // [ngroups][B][G]
    double2* __restrict__ part_r,  // [n_ig_tiles][B][ngroups * kTY]
    double sx2)                    // screened-exchange cutoff, sexcut^2 (0 = off)
{
  __shared__ double2 s_a[kTY][kTX];
  __shared__ double2 s_r[kTY][kTX];
  const bool x_nonneg = flags[0] == 0;
  const double wabs2_pf = pf_wabs2_min(flags);   // the partial fractions' bound (gpp_device.cuh)
  const int64_t ntiles = static_cast<int64_t>(ngroups) * n_ig_tiles;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // G-vector tile slowest, so the CTAs running together share one slab of aqsntemp
    const int64_t igt = t / ngroups;
    const int gl = static_cast<int>(t - igt * ngroups);       // group within the batch
    const int64_t p = (group0 + gl) * kTY + ty;
    const int64_t ig = igt * kTX + tx;
    const bool col_ok = p < P && colg[p] >= 0;
    const bool live = col_ok && ig < G;
    double2 w = make_double2(0.5, 1.0);  // inert lane: finite terms, zero weight
    double2 I = make_double2(0.0, 0.0);
    if (live) {
      w = ldg2(wt + p * G + ig);
      I = ldg2(eps + p * G + ig);
    }
    const double wr = w.x, wi = w.y;
    const double wi2 = wi * wi;
    const double wabs2 = fma(wr, wr, wi2);
    const double mw2r = -fma(wr, wr, -wi2);
    const double w2i = 2.0 * wr * wi;
    const double2 Iw = cmul(I, w);
    const bool fast_lane = wr >= 0.0 && gt_nonneg(wabs2, kFastWabs2Lo) &&
                           lt_nonneg(wabs2, kFastWabs2Hi) && !lt_nonneg(wabs2, wabs2_pf);
    const bool fast = __all_sync(0xffffffffu, fast_lane) && x_nonneg;
    const double2* an_ptr = aqsn + (ig < G ? ig : 0);
    const double2* am_ptr = am + (col_ok ? p : 0) * B;
    double2 gw = make_double2(0.0, 0.0), gI = make_double2(0.0, 0.0);
    // bands [0, nocc) enter asxtemp too; OCC is a template parameter of the band body
    auto band = [&](int b, auto occ_tag) {
      constexpr bool OCC = decltype(occ_tag)::value;
      const double2 an = (ig < G) ? ldg2(an_ptr + static_cast<int64_t>(b) * G) : make_double2(0.0, 0.0);
      const double2 amv = col_ok ? ldg2(am_ptr + b) : make_double2(0.0, 0.0);
      double2 GI = make_double2(0.0, 0.0), GW = make_double2(0.0, 0.0);
      const BwdBand* e = bt + static_cast<int64_t>(b) * W;
      if (fast)
        bwd_terms_fast<W, OCC>(e, wr, wi, wi2, GI, GW);
      else
        bwd_terms<W, OCC>(e, wr, wi, wi2, wabs2, mw2r, w2i, w, sx2, GI, GW);
      // sum_b M w GI and sum_b M I GW: w and I are the thread's constants, applied at the end
      const double2 M = cmul(amv, an);
      cmac(gI, M, GI);
      cmac(gw, M, GW);
      const double2 Q = live ? cmul(Iw, GI) : make_double2(0.0, 0.0);
      s_a[ty][tx] = cmul(amv, Q);
      s_r[ty][tx] = cmul(an, Q);
      __syncthreads();
      tile_reduce(s_a, s_r);
      if (ty == 0 && ig < G)
        part_n[(static_cast<int64_t>(gl) * B + b) * G + ig] = s_a[0][tx];
      if (tx == 0)
        part_r[(igt * B + b) * (static_cast<int64_t>(ngroups) * kTY) + gl * kTY + ty] = s_r[ty][0];
      __syncthreads();
    };
    for (int b = 0; b < nocc; ++b) band(b, BoolTag<true>());
    for (int b = nocc; b < B; ++b) band(b, BoolTag<false>());
    gI = cmul(w, gI);
    gw = cmul(I, gw);
    if (live) {
      if (grad_w) grad_w[p * G + ig] = make_double2(gw.x, -gw.y);
      if (grad_I) grad_I[p * G + ig] = make_double2(gI.x, -gI.y);
    } else if (p < P && ig < G) {
      if (grad_w) grad_w[p * G + ig] = make_double2(0.0, 0.0);
      if (grad_I) grad_I[p * G + ig] = make_double2(0.0, 0.0);
    }
  }
}

// grad_aqsn[b][ig] (+)= conj(sum over the batch's groups, in order); rtot[b][p] = sum over
// ig tiles, in order, for the batch's columns.
__global__ void gpp_bwd_finish_batch_kernel(int64_t B, int64_t G, int64_t P, int64_t group0,
                                            int ngroups, int64_t n_ig_tiles, bool first,
                                            const double2* __restrict__ part_n,
                                            const double2* __restrict__ part_r,
                                            double2* __restrict__ grad_n, double2* __restrict__ rtot) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int64_t i = tid; i < B * G; i += stride) {
    double2 s = make_double2(0.0, 0.0);
    for (int gl = 0; gl < ngroups; ++gl) {
      const double2 v = part_n[static_cast<int64_t>(gl) * B * G + i];
      s.x += v.x;
      s.y += v.y;
    }
    if (grad_n) {
      double2 o = first ? make_double2(0.0, 0.0) : grad_n[i];
      grad_n[i] = make_double2(o.x + s.x, o.y - s.y);
    }
  }
  const int64_t ncols = static_cast<int64_t>(ngroups) * kTY;
  for (int64_t i = tid; i < B * ncols; i += stride) {
    const int64_t b = i / ncols, c = i - b * ncols;
    const int64_t p = group0 * kTY + c;
    if (p >= P) continue;
    double2 s = make_double2(0.0, 0.0);
    for (int64_t it = 0; it < n_ig_tiles; ++it) {
      const double2 v = part_r[(it * B + b) * ncols + c];
      s.x += v.x;
      s.y += v.y;
    }
    rtot[b * P + p] = s;
  }
}

// grad_aqsm[b][g] = vcoul[g] * sum over columns p with g(p) = g, in increasing p; zero for
// global columns no column reaches. One thread per (b, g).
__global__ void gpp_bwd_aqsm_kernel(int64_t B, int64_t G, int64_t P, const int* __restrict__ colg,
                                    const double* __restrict__ vcoul,
                                    const double2* __restrict__ rtot, double2* __restrict__ grad_m) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < B * G;
       i += stride)
    grad_m[i] = make_double2(0.0, 0.0);
  // second phase handled by gpp_bwd_aqsm_scatter_kernel (after this kernel completes)
}

__global__ void gpp_bwd_aqsm_scatter_kernel(int64_t B, int64_t P, int64_t G,
                                            const int* __restrict__ colg,
                                            const double* __restrict__ vcoul,
                                            const double2* __restrict__ rtot,
                                            double2* __restrict__ grad_m) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < B * P;
       i += stride) {
    const int64_t b = i / P, p = i - b * P;
    const int g = colg[p];
    if (g < 0) continue;
    bool first = true;
    for (int64_t q = 0; q < p; ++q)
      if (colg[q] == g) {
        first = false;
        break;
      }
    if (!first) continue;  // the first column with this g sums all of them, in order
    double2 s = make_double2(0.0, 0.0);
    for (int64_t q = p; q < P; ++q)
      if (colg[q] == g) {
        const double2 v = rtot[b * P + q];
        s.x += v.x;
        s.y += v.y;
      }
    const double vc = vcoul[g];
    grad_m[b * G + g] = make_double2(vc * s.x, vc * s.y);
  }
}

template <int W>
const void* bwd_fn() {
  return reinterpret_cast<const void*>(&gpp_bwd_kernel<W>);
}

const void* bwd_kernel_ptr(int nw) {
  switch (nw) {
    case 1: return bwd_fn<1>();
    case 2: return bwd_fn<2>();
    case 3: return bwd_fn<3>();
    case 4: return bwd_fn<4>();
    case 5: return bwd_fn<5>();
    case 6: return bwd_fn<6>();
    case 7: return bwd_fn<7>();
    case 8: return bwd_fn<8>();
    default: return nullptr;
  }
}

int grid_for(int64_t work) {
  int64_t b = (work + 255) / 256;
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return static_cast<int>(b);
}

}  // namespace

int bwd_blocks_per_sm(int nw) {
  const void* fn = bwd_kernel_ptr(nw);
  if (!fn) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kTX * kTY, 0) != cudaSuccess) return 0;
  return n;
}

int64_t bwd_groups(int64_t P) { return (P + kTY - 1) / kTY; }
int bwd_tile_ig() { return kTX; }
int bwd_tile_cols() { return kTY; }

cudaError_t launch_bwd(const gpp_problem& p, int occ_mode, double ach_scale, double sx2,
                       const BwdPlan& plan, char* ws, const gpp_c128* g_ach,
                       const gpp_c128* g_asx, const gpp_grads& out, cudaStream_t s) {
  const int64_t B = p.number_bands, G = p.ncouls, P = p.ngpown;
  const int W = static_cast<int>(p.nw);
  int64_t nocc = B;
  if (occ_mode == GPP_OCC_OCCUPIED) nocc = p.nvband < B ? p.nvband : B;
  BwdBand* bt = reinterpret_cast<BwdBand*>(ws + plan.off_bwd_bt);
  gpp_bwd_prep_kernel<<<grid_for(B * W), 256, 0, s>>>(B, W, p.wx_array,
                                                      reinterpret_cast<const double2*>(g_ach),
                                                      reinterpret_cast<const double2*>(g_asx),
                                                      ach_scale, bt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double2* am = reinterpret_cast<const double2*>(ws + plan.fwd.off_am);
  const int* colg = reinterpret_cast<const int*>(ws + plan.fwd.off_colvalid);
  const int* flags = reinterpret_cast<const int*>(ws + plan.fwd.off_flags);
  double2* part_n = reinterpret_cast<double2*>(ws + plan.off_part_n);
  double2* part_r = reinterpret_cast<double2*>(ws + plan.off_part_r);
  double2* rtot = reinterpret_cast<double2*>(ws + plan.off_rtot);
  const int64_t ngroups_total = bwd_groups(P);
  const int64_t n_ig_tiles = (G + kTX - 1) / kTX;
  const dim3 block(kTX, kTY);
  for (int64_t g0 = 0; g0 < ngroups_total; g0 += plan.batch_groups) {
    const int ng = static_cast<int>(ngroups_total - g0 < plan.batch_groups ? ngroups_total - g0
                                                                            : plan.batch_groups);
    const int64_t ntiles = ng * n_ig_tiles;
    int grid = static_cast<int>(ntiles < plan.max_grid ? ntiles : plan.max_grid);
#define GPP_BWD_LAUNCH(WV)                                                                        \
  gpp_bwd_kernel<WV><<<grid, block, 0, s>>>(                                                      \
      static_cast<int>(B), G, P, static_cast<int>(nocc), g0, ng, n_ig_tiles,                      \
      reinterpret_cast<const double2*>(p.aqsntemp), reinterpret_cast<const double2*>(p.I_eps_array), \
      reinterpret_cast<const double2*>(p.wtilde_array), am, bt, colg, flags,                      \
      reinterpret_cast<double2*>(out.wtilde_array), reinterpret_cast<double2*>(out.I_eps_array),  \
      part_n, part_r, sx2)
    switch (W) {
      case 1: GPP_BWD_LAUNCH(1); break;
      case 2: GPP_BWD_LAUNCH(2); break;
      case 3: GPP_BWD_LAUNCH(3); break;
      case 4: GPP_BWD_LAUNCH(4); break;
      case 5: GPP_BWD_LAUNCH(5); break;
      case 6: GPP_BWD_LAUNCH(6); break;
      case 7: GPP_BWD_LAUNCH(7); break;
      case 8: GPP_BWD_LAUNCH(8); break;
      default: return cudaErrorInvalidValue;
    }
#undef GPP_BWD_LAUNCH
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    gpp_bwd_finish_batch_kernel<<<grid_for(B * G), 256, 0, s>>>(
        B, G, P, g0, ng, n_ig_tiles, g0 == 0, part_n, part_r,
        reinterpret_cast<double2*>(out.aqsntemp), rtot);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (out.aqsmtemp) {
    gpp_bwd_aqsm_kernel<<<grid_for(B * G), 256, 0, s>>>(B, G, P, colg, p.vcoul, rtot,
                                                        reinterpret_cast<double2*>(out.aqsmtemp));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    gpp_bwd_aqsm_scatter_kernel<<<grid_for(B * P), 256, 0, s>>>(
        B, P, G, colg, p.vcoul, rtot, reinterpret_cast<double2*>(out.aqsmtemp));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace gpp
