// The main GPP sum: one persistent launch over the tiles of one or many instances (a
// single gpp_sigma call is a batch of one).
//
// Work unit: a tile = one local column p of one instance x (threads * ig_per_thread)
// G-vectors, all bands. Tiles of all instances form one list, ordered by instance band count
// (largest first, so the longest tiles start first and the tail is short); within an
// instance the G-vector tile varies slowest, so the tiles running at the same time share
// the same slab of aqsntemp (all bands x the tile's G-vectors) through L2. CTAs of a
// persistent grid take tiles from an atomic counter; the counter only schedules, and every
// tile writes its own partial slot, so the result does not depend on which CTA ran which
// tile. A per-instance kernel then sums the instance's tile partials in tile order. The
// per-tile arithmetic is the single-instance kernels' (gpp_terms_f64.cuh / gpp_terms_f32.cuh).

#include <cuda_runtime.h>

#include "gpp_device.cuh"
#include "gpp_internal.h"
#include "gpp_terms_f32.cuh"
#include "gpp_terms_f64.cuh"

namespace gpp {

namespace {

// Band count from which the FP32-bulk kernel sorts a tile's G-vectors by Re w.
constexpr int kSortBands = 128;

// Smallest power of two >= n (n >= 1).
__host__ __device__ inline int pow2_ceil(int n) {
  int k = 1;
  while (k < n) k <<= 1;
  return k;
}

// Sorts every aligned segment key[s seg, (s + 1) seg) of key[0, n) and permutes idx with
// it (n and seg powers of two, seg <= n; every thread of the block takes part): even
// segments ascending, odd ones descending (seg = n: all of it ascending). The first stages
// of a bitonic network: deterministic for fixed keys, and a permutation of idx within each
// segment whatever the keys (NaN compares false and never swaps).
__device__ inline void bitonic_sort(float* key, int* idx, int n, int seg) {
  for (int k = 2; k <= seg; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const float a = key[i], b = key[l];
          if ((i & k) == 0 ? a > b : a < b) {
            key[i] = b;
            key[l] = a;
            const int t = idx[i];
            idx[i] = idx[l];
            idx[l] = t;
          }
        }
      }
      __syncthreads();
    }
  }
}

// The FP32-bulk kernel's general path for one (igp, ig) pair: the FP64 band loop, folded
// into the thread's tile pairs. Not inlined: its FP64 accumulators would otherwise count
// against the register budget of the FP32 band loop, which it shares a kernel with (and
// the warps that take it are rare).
template <int W>
__device__ __noinline__ void f32_general_pair(int B, int64_t G, int nocc,
                                              const double2* __restrict__ aqsn,
                                              const double2* __restrict__ am,
                                              const BandEntry* __restrict__ bt, bool live,
                                              double wr, double wi, double Iwr, double Iwi,
                                              double sx2, float4* tp) {
  double a[4 * W];
#pragma unroll
  for (int k = 0; k < 4 * W; ++k) a[k] = 0.0;
  band_loop<W, false>(B, G, nocc, aqsn, am, bt, live, wr, wi, Iwr, Iwi, sx2, a);
#pragma unroll
  for (int qd = 0; qd < W; ++qd) {
    float4 th = tp[qd], tl = tp[W + qd];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double v = a[4 * qd + i];
      const float h = static_cast<float>(v);
      pair_add(quad_elem(th, i), quad_elem(tl, i), h, static_cast<float>(v - static_cast<double>(h)));
    }
    tp[qd] = th;
    tp[W + qd] = tl;
  }
}

// Tile partials: FP64 sums (double) for GPP_FP64; compensated FP32 pairs (float2, hi + lo)
// for GPP_FP32_BULK, so that its main kernel needs no FP64 arithmetic outside the rare
// exact-decision and near-pole branches and the once-per-pair I w. Both are 8 bytes per
// value. The FP32-bulk instantiation is held to 72 registers per thread: with its shared
// memory (the compensated pairs) that is 7 CTAs of 128 threads per SM either way, and on
// GB300 (nw = 3, benchmark instance) its main kernel ran 111.2 ms at 64 registers (spilled
// values reloaded in the band loop), 104.5 ms at 72 and 105.9 ms at 80.
#ifndef GPP_F32_MAXNREG
#define GPP_F32_MAXNREG 72
#endif
template <int W, bool F32>
__device__ __forceinline__ void batched_body(const BatchInst* __restrict__ inst, int ninst,
                                             int64_t t_begin, int64_t ntiles, int igpt,
                                             unsigned long long* counter,
                                             double* __restrict__ partials) {
  __shared__ double red[(256 / 32) * 4 * kMaxNw];
  __shared__ long long s_t;
  __shared__ const BandEntry* s_bt64;  // FP32-bulk: the FP64 band table, for the exact path
  // FP32-bulk: the threads' slots (F32Slots: band compensated pairs, FP64 wtilde; (8 W + 4)
  // floats per thread), then the tile's G-vector positions in sorted order
  // (int[pow2_ceil(blockDim.x * igpt)]); the sort keys (float, as many) alias the start of
  // the slots, which are written only after the sort, and the slot area is at least as long
  // as the keys (dynamic shared memory of batched_smem_bytes)
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float* const s_slots = reinterpret_cast<float*>(dyn_smem);
  const int tile_n = blockDim.x * igpt;
  const int sort_n = F32 ? pow2_ceil(tile_n) : 0;
  float* const s_key = s_slots;
  int* const s_pos = reinterpret_cast<int*>(
      s_slots + max(F32Slots<W>::kFloats * static_cast<int>(blockDim.x), sort_n));
  // FP32-bulk: the thread's tile sums as compensated pairs (hi quads [0, W), lo quads
  // [W, 2W)), in local memory (the address goes to the non-inlined fold and general-path
  // functions); touched once per (igp, ig) pair
  float4 tpair[2 * W];
  for (;;) {
    if (threadIdx.x == 0) s_t = t_begin + static_cast<long long>(atomicAdd(counter, 1ULL));
    __syncthreads();
    const int64_t t = s_t;
    __syncthreads();
    if (t >= ntiles) break;
    int ilo = 0, ihi = ninst - 1;  // instance holding tile t (tile ranges are sorted)
    while (ilo < ihi) {
      const int mid = (ilo + ihi) >> 1;
      if (__ldg(&inst[mid].tile_end) > t)
        ihi = mid;
      else
        ilo = mid + 1;
    }
    const BatchInst& d = inst[ilo];
    const int B = d.B, nocc = d.nocc;
    const int64_t G = d.G;
    const int64_t local = t - d.tile0;
    const int64_t igt = local / d.P;
    const int64_t p = local - igt * d.P;
    const bool col_ok = d.colg[p] >= 0;
    const bool x_fast = d.flags[0] == 0 && (!F32 || d.flags[2] == 0);
    // FP64: the partial fractions' bound on x / |w| (gpp_device.cuh)
    const double wabs2_pf = F32 ? 0.0 : pf_wabs2_min(d.flags);
    double acc[4 * W];                 // FP64 sums (GPP_FP64)
#pragma unroll
    for (int k = 0; k < 4 * W; ++k) acc[k] = 0.0;
    if (F32) {
      if (threadIdx.x == 0) s_bt64 = d.bt;
      // With at least kSortBands bands, the G-vectors of each pass over the tile (blockDim.x
      // of them, when that is a power of two; else the whole tile) are taken in order of
      // Re w, so that the 32 of a warp (consecutive in that order) span a narrow range of
      // Re w and most frequencies fall outside it (the far-from-threshold path). Sorting
      // within a pass keeps a warp's aqsntemp loads inside the pass's contiguous slice
      // (blockDim.x x 8 bytes per band). With fewer bands the sort and the scattered loads
      // cost more than they save. The sum does not depend on which thread takes which
      // G-vector; inert positions (past G, dead column) carry +inf keys.
      const bool sort = B >= kSortBands;
      for (int q = threadIdx.x; q < sort_n; q += blockDim.x) {
        const int64_t ig = igt * tile_n + q;
        float key = __int_as_float(0x7f800000);
        if (sort && q < tile_n && ig < G && col_ok) {
          key = static_cast<float>(__ldg(&d.wt[p * G + ig].x));
          key = key == key ? key : 0.0f;  // a NaN must still sort among the live positions
        }
        s_key[q] = key;
        s_pos[q] = q;
      }
      __syncthreads();
      if (sort) {
        const int nt = blockDim.x;
        bitonic_sort(s_key, s_pos, sort_n, (nt & (nt - 1)) == 0 ? nt : sort_n);
      }
      __syncthreads();  // the keys' space becomes the threads' slots
#pragma unroll
      for (int k = 0; k < 2 * W; ++k) tpair[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int j = 0; j < igpt; ++j) {
      // F32: a padding position (>= tile_n, key +inf like an inert one) can sort into the
      // first tile_n slots when the whole tile is sorted; it is inert
      const int q = F32 ? s_pos[j * blockDim.x + threadIdx.x] : 0;
      const int64_t ig = F32 ? igt * tile_n + q : (igt * igpt + j) * blockDim.x + threadIdx.x;
      const bool live = (!F32 || q < tile_n) && ig < G && col_ok;
      double2 w = make_double2(0.5, 1.0);  // inert lane: finite terms, zero weight
      if (live) w = ldg2(d.wt + p * G + ig);
      const double wabs2 = fma(w.x, w.x, w.y * w.y);
      const bool fast_lane = w.x >= 0.0 && gt_nonneg(wabs2, kFastWabs2Lo) &&
                             lt_nonneg(wabs2, kFastWabs2Hi) && !lt_nonneg(wabs2, wabs2_pf);
      const bool fast = __all_sync(0xffffffffu, fast_lane) && x_fast;
      if (F32 && fast) {
        band_loop_f32<W>(B, G, nocc, d.aqsn32 + (live ? ig : 0), d.am32 + p * B, d.bt32,
                         &s_bt64, w, live, s_slots);
        // I w in FP64 once per pair (w re-read from the thread's slot, I from memory, so
        // that neither stays in registers through the band loop)
        const volatile double* ws = reinterpret_cast<volatile double*>(F32Slots<W>::w64(s_slots));
        const double2 wv = make_double2(ws[0], ws[1]);
        double2 I = make_double2(0.0, 0.0);
        if (live) I = ldg2(d.eps + p * G + ig);
        fold_band_sums<W>(s_slots, tpair, make_double2(fma(I.x, wv.x, -I.y * wv.y),
                                                       fma(I.x, wv.y, I.y * wv.x)));
        continue;
      }
      double2 I = make_double2(0.0, 0.0);
      if (live) I = ldg2(d.eps + p * G + ig);
      const double Iwr = fma(I.x, w.x, -I.y * w.y);
      const double Iwi = fma(I.x, w.y, I.y * w.x);
      if (F32) {  // the general path in FP64, folded into the tile pairs
        f32_general_pair<W>(B, G, nocc, d.aqsn + (live ? ig : 0), d.am + p * B, d.bt, live,
                            w.x, w.y, Iwr, Iwi, d.sx2, tpair);
      } else if (fast) {
        band_loop<W, true>(B, G, nocc, d.aqsn + (live ? ig : 0), d.am + p * B, d.bt, live,
                           w.x, w.y, Iwr, Iwi, 0.0, acc);
      } else {
        band_loop<W, false>(B, G, nocc, d.aqsn + (live ? ig : 0), d.am + p * B, d.bt, live,
                            w.x, w.y, Iwr, Iwi, d.sx2, acc);
      }
    }
    if (F32) {
      float hi[4 * W], lo[4 * W];
#pragma unroll
      for (int qd = 0; qd < W; ++qd) {
        float4 th = tpair[qd], tl = tpair[W + qd];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          hi[4 * qd + i] = quad_elem(th, i);
          lo[4 * qd + i] = quad_elem(tl, i);
        }
      }
      block_pairs<4 * W>(hi, lo, reinterpret_cast<float2*>(red),
                         reinterpret_cast<float2*>(partials) + t * 4 * W);
    }
    else
      block_partials<4 * W>(acc, red, partials + t * 4 * W);
  }
}

// The two instantiations of the main kernel. FP64: one 256-thread CTA's worth of registers
// per SM at most (the FP64 band loop takes ~160 registers). FP32-bulk: held to
// GPP_F32_MAXNREG registers (80 for nw > 5, whose band loop would spill at fewer).
template <int W>
__global__ void __launch_bounds__(256, 1)
    gpp_batched_kernel_f64(const BatchInst* __restrict__ inst, int ninst, int64_t t_begin,
                           int64_t ntiles, int igpt, unsigned long long* counter,
                           double* __restrict__ partials) {
  batched_body<W, false>(inst, ninst, t_begin, ntiles, igpt, counter, partials);
}

template <int W>
__global__ void __launch_bounds__(256) __maxnreg__(W <= 5 ? GPP_F32_MAXNREG : 80)
    gpp_batched_kernel_f32(const BatchInst* __restrict__ inst, int ninst, int64_t t_begin,
                           int64_t ntiles, int igpt, unsigned long long* counter,
                           double* __restrict__ partials) {
  batched_body<W, true>(inst, ninst, t_begin, ntiles, igpt, counter, partials);
}

// One CTA per instance: the instance's tile partials summed in tile order, then a tree.
template <bool F32>
__global__ void __launch_bounds__(256) gpp_batched_reduce_kernel(const BatchInst* __restrict__ inst,
                                                                 int nv,
                                                                 const double* __restrict__ part) {
  __shared__ double s[256];
  const BatchInst& d = inst[blockIdx.x];
  const int64_t n = d.tile_end - d.tile0;
  for (int k = 0; k < nv; ++k) {
    double v = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += 256) {
      if (F32) {
        const float2 q = reinterpret_cast<const float2*>(part)[(d.tile0 + j) * nv + k];
        v += static_cast<double>(q.x) + static_cast<double>(q.y);
      } else {
        v += part[(d.tile0 + j) * nv + k];
      }
    }
    s[threadIdx.x] = v;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int iw = k / 4, c = k % 4;
      if (c < 2)
        reinterpret_cast<double*>(d.ach)[2 * iw + c] = s[0] * d.ach_scale;
      else
        reinterpret_cast<double*>(d.asx)[2 * iw + c - 2] = s[0];
    }
    __syncthreads();
  }
}

template <int W, bool F32>
const void* batched_fn() {
  return F32 ? reinterpret_cast<const void*>(&gpp_batched_kernel_f32<W>)
             : reinterpret_cast<const void*>(&gpp_batched_kernel_f64<W>);
}

const void* batched_kernel_ptr(int nw, bool f32) {
  switch (nw) {
    case 1: return f32 ? batched_fn<1, true>() : batched_fn<1, false>();
    case 2: return f32 ? batched_fn<2, true>() : batched_fn<2, false>();
    case 3: return f32 ? batched_fn<3, true>() : batched_fn<3, false>();
    case 4: return f32 ? batched_fn<4, true>() : batched_fn<4, false>();
    case 5: return f32 ? batched_fn<5, true>() : batched_fn<5, false>();
    case 6: return f32 ? batched_fn<6, true>() : batched_fn<6, false>();
    case 7: return f32 ? batched_fn<7, true>() : batched_fn<7, false>();
    case 8: return f32 ? batched_fn<8, true>() : batched_fn<8, false>();
    default: return nullptr;
  }
}

}  // namespace

size_t batched_smem_bytes(int threads, int nw, bool f32, int igpt) {
  // F32Slots<nw>::kFloats floats per thread (at least as many as the sort keys, which alias
  // them), then the sorted positions
  if (!f32) return 0;
  const size_t sort_n = static_cast<size_t>(pow2_ceil(threads * igpt));
  const size_t slots = static_cast<size_t>(threads) * (8 * nw + 4);
  return (slots > sort_n ? slots : sort_n) * sizeof(float) + sort_n * sizeof(int);
}

// A CTA whose static + dynamic shared memory exceeds 48 KB (nw >= 6 at 256 threads) must
// opt in; the kernel's static part (the reduction buffer) is below 4 KB. Called at plan
// time, outside any stream capture.
cudaError_t batched_prepare(int threads, int nw, bool f32, int igpt) {
  const void* fn = batched_kernel_ptr(nw, f32);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = batched_smem_bytes(threads, nw, f32, igpt);
  if (smem + 4096 <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(smem));
}

int batched_blocks_per_sm(int threads, int nw, bool f32, int igpt) {
  const void* fn = batched_kernel_ptr(nw, f32);
  if (!fn) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads,
                                                    batched_smem_bytes(threads, nw, f32, igpt)) !=
      cudaSuccess)
    return 0;
  return n;
}

cudaError_t launch_batched_main(const BatchInst* inst, int ninst, int64_t ntiles, int nw,
                                bool f32, int grid, int threads, int igpt,
                                unsigned long long* counter, double* partials, cudaStream_t s,
                                int64_t t_begin) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const size_t smem = batched_smem_bytes(threads, nw, f32, igpt);
#define GPP_BATCHED_LAUNCH(WV)                                                                    \
  if (f32)                                                                                        \
    gpp_batched_kernel_f32<WV><<<grid, threads, smem, s>>>(inst, ninst, t_begin, ntiles, igpt,    \
                                                           counter, partials);                    \
  else                                                                                            \
    gpp_batched_kernel_f64<WV><<<grid, threads, 0, s>>>(inst, ninst, t_begin, ntiles, igpt,       \
                                                        counter, partials)
  switch (nw) {
    case 1: GPP_BATCHED_LAUNCH(1); break;
    case 2: GPP_BATCHED_LAUNCH(2); break;
    case 3: GPP_BATCHED_LAUNCH(3); break;
    case 4: GPP_BATCHED_LAUNCH(4); break;
    case 5: GPP_BATCHED_LAUNCH(5); break;
    case 6: GPP_BATCHED_LAUNCH(6); break;
    case 7: GPP_BATCHED_LAUNCH(7); break;
    case 8: GPP_BATCHED_LAUNCH(8); break;
    default: return cudaErrorInvalidValue;
  }
#undef GPP_BATCHED_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_batched_reduce(const BatchInst* inst, int ninst, int nw, bool f32,
                                  const double* partials, cudaStream_t s) {
  if (f32)
    gpp_batched_reduce_kernel<true><<<ninst, 256, 0, s>>>(inst, 4 * nw, partials);
  else
    gpp_batched_reduce_kernel<false><<<ninst, 256, 0, s>>>(inst, 4 * nw, partials);
  return cudaGetLastError();
}

}  // namespace gpp
