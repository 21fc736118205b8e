// C-ABI entry points of libgpp (declared in include/gpp.h): argument validation,
// workspace layout and kernel launches. No entry point allocates device memory.

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "gpp.h"
#include "gpp_device.cuh"
#include "gpp_diag.h"
#include "gpp_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

// Host-side fault injection (gpp_diag_inject_cuda_failure): a countdown of checked CUDA
// calls on this host thread; the call at which it reaches zero reports failure after it has
// been made.
thread_local int g_inject_countdown = 0;
thread_local bool g_injected = false;

int cuda_fail(cudaError_t e, const char* what) {
  const bool inj = g_injected;
  g_injected = false;
  return fail(GPP_ERR_CUDA, "%s: %s (%s)%s", what, cudaGetErrorName(e), cudaGetErrorString(e),
              inj ? " [injected by gpp_diag_inject_cuda_failure]" : "");
}

cudaError_t checked(cudaError_t e) { return gpp::checked(e); }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

gpp_options defaults() {
  gpp_options o;
  memset(&o, 0, sizeof(o));
  o.precision = GPP_FP64;
  o.occ_mode = GPP_OCC_ALL;
  return o;
}

bool degenerate(const gpp_problem& p) {
  return p.number_bands == 0 || p.ngpown == 0 || p.ncouls == 0;
}

int check_options(const gpp_options& o) {
  if (o.precision != GPP_FP64 && o.precision != GPP_FP32_BULK)
    return fail(GPP_ERR_BAD_OPTION, "precision %d is not GPP_FP64 or GPP_FP32_BULK", o.precision);
  if (o.occ_mode != GPP_OCC_ALL && o.occ_mode != GPP_OCC_OCCUPIED)
    return fail(GPP_ERR_BAD_OPTION, "occ_mode %d is not GPP_OCC_ALL or GPP_OCC_OCCUPIED", o.occ_mode);
  if (o.block_threads != 0 &&
      (o.block_threads < 64 || o.block_threads > 256 || o.block_threads % 32 != 0))
    return fail(GPP_ERR_BAD_OPTION, "block_threads %d must be 0 or a multiple of 32 in [64, 256]",
                o.block_threads);
  if (o.blocks_per_sm < 0 || o.blocks_per_sm > 64)
    return fail(GPP_ERR_BAD_OPTION, "blocks_per_sm %d must be in [0, 64]", o.blocks_per_sm);
  if (o.debug_checks != 0 && o.debug_checks != 1)
    return fail(GPP_ERR_BAD_OPTION, "debug_checks must be 0 or 1");
  if (o.ig_per_thread < 0 || o.ig_per_thread > 8)
    return fail(GPP_ERR_BAD_OPTION, "ig_per_thread %d must be in [0, 8]", o.ig_per_thread);
  if (o.physics & ~(GPP_PHYS_CH_HALF | GPP_PHYS_SX_CUTOFF))
    return fail(GPP_ERR_BAD_OPTION, "physics %d has unknown bits", o.physics);
  if ((o.physics & GPP_PHYS_SX_CUTOFF) && !(o.sexcut > 0.0 && o.sexcut < 1e300))
    return fail(GPP_ERR_BAD_OPTION, "sexcut %g must be positive and finite", o.sexcut);
  if (o.reserved != 0) return fail(GPP_ERR_BAD_OPTION, "the reserved option field must be 0");
  return GPP_OK;
}

int check_sizes(const gpp_problem& p) {
  if (p.number_bands < 0 || p.nvband < 0 || p.ncouls < 0 || p.ngpown < 0)
    return fail(GPP_ERR_BAD_SIZE, "negative size (number_bands %lld nvband %lld ncouls %lld ngpown %lld)",
                (long long)p.number_bands, (long long)p.nvband, (long long)p.ncouls,
                (long long)p.ngpown);
  if (p.nw < 1 || p.nw > GPP_MAX_NW)
    return fail(GPP_ERR_BAD_SIZE, "nw %lld outside [1, %d]", (long long)p.nw, GPP_MAX_NW);
  if (p.number_bands > INT32_MAX || p.ncouls >= INT32_MAX || p.ngpown > INT32_MAX)
    return fail(GPP_ERR_BAD_SIZE, "sizes must fit 32-bit indices");
  return GPP_OK;
}

// Pointers the forward pass reads for this precision; complex arrays 16- or 8-byte aligned.
int check_pointers(const gpp_problem& p, int precision, bool outputs = true) {
  if (outputs) {
    if (!p.achtemp || !p.asxtemp) return fail(GPP_ERR_NULL_PTR, "achtemp and asxtemp must be non-NULL");
    if (!aligned(p.achtemp, 16) || !aligned(p.asxtemp, 16))
      return fail(GPP_ERR_NULL_PTR, "achtemp / asxtemp must be 16-byte aligned");
  }
  if (degenerate(p)) return GPP_OK;
  struct {
    const void* ptr;
    const char* name;
    size_t align;
  } req[] = {{p.aqsmtemp, "aqsmtemp", 16},     {p.aqsntemp, "aqsntemp", 16},
             {p.I_eps_array, "I_eps_array", 16}, {p.wtilde_array, "wtilde_array", 16},
             {p.vcoul, "vcoul", 8},             {p.inv_igp_index, "inv_igp_index", 4},
             {p.indinv, "indinv", 4},           {p.wx_array, "wx_array", 8}};
  for (auto& r : req) {
    if (!r.ptr) return fail(GPP_ERR_NULL_PTR, "%s is NULL", r.name);
    if (!aligned(r.ptr, r.align)) return fail(GPP_ERR_NULL_PTR, "%s is not %zu-byte aligned", r.name, r.align);
  }
  if (precision == GPP_FP32_BULK && p.aqsntemp_c64 && !aligned(p.aqsntemp_c64, 8))
    return fail(GPP_ERR_NULL_PTR, "aqsntemp_c64 is not 8-byte aligned");
  return GPP_OK;
}

// Default G-vectors per thread of a tile. On GB300 (benchmark instance, 128 threads) the
// FP32-bulk main kernel ran 93.6 / 92.6 / 95.3 / 94.2 / 94.9 ms at 1 / 2 / 3 / 4 / 8.
int default_igpt(int precision) { return precision == GPP_FP32_BULK ? 2 : 4; }

// Workspace layout of one instance. The gather segments come first; unless `gather_only`
// (instances of a batched plan, the adjoint), the descriptor, tile counter and per-tile
// partials of the main kernel follow.
int make_plan(const gpp_problem& p, const gpp_options& o, gpp::FwdPlan* plan,
              bool gather_only = false) {
  gpp::FwdPlan pl;
  pl.nw = static_cast<int>(p.nw);
  const bool f32 = o.precision == GPP_FP32_BULK;
  pl.threads = o.block_threads ? o.block_threads : 128;
  pl.igpt = o.ig_per_thread ? o.ig_per_thread : default_igpt(o.precision);
  if (degenerate(p)) {
    *plan = pl;
    return GPP_OK;
  }
  size_t off = 0;
  pl.off_flags = off;
  off = gpp::align_up(off + gpp::kFlagBytes);
  pl.off_colvalid = off;
  off = gpp::align_up(off + static_cast<size_t>(p.ngpown) * sizeof(int));
  pl.off_bt = off;
  off = gpp::align_up(off + static_cast<size_t>(p.number_bands) * p.nw * 4 * sizeof(double));
  pl.off_am = off;
  off = gpp::align_up(off + static_cast<size_t>(p.ngpown) * p.number_bands * 2 * sizeof(double));
  if (f32) {
    pl.off_bt32 = off;
    off = gpp::align_up(off + static_cast<size_t>(p.number_bands) *
                                  (2 * ((p.nw + 4) / 4)) * 16);  // f32_band_quads
    pl.off_am32 = off;
    off = gpp::align_up(off + static_cast<size_t>(p.ngpown) * p.number_bands * 2 * sizeof(float));
    if (!p.aqsntemp_c64) {  // the library makes the complex64 copy of aqsntemp
      pl.convert_c64 = true;
      pl.off_aqsn32 = off;
      off = gpp::align_up(off + static_cast<size_t>(p.number_bands) * p.ncouls * 2 * sizeof(float));
    }
  }
  pl.gather_total = off;
  if (!gather_only) {
    int dev = 0, sms = 0;
    cudaError_t e = checked(cudaGetDevice(&dev));
    if (e == cudaSuccess) e = checked(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (e == cudaSuccess) e = gpp::batched_prepare(pl.threads, pl.nw, f32, pl.igpt);
    if (e != cudaSuccess) return cuda_fail(e, "querying the device");
    int bps = o.blocks_per_sm ? o.blocks_per_sm
                              : gpp::batched_blocks_per_sm(pl.threads, pl.nw, f32, pl.igpt);
    if (bps <= 0) return fail(GPP_ERR_CUDA, "occupancy query failed for %d threads", pl.threads);
    const int64_t tile_ig = static_cast<int64_t>(pl.threads) * pl.igpt;
    pl.n_ig_tiles = (p.ncouls + tile_ig - 1) / tile_ig;
    pl.ntiles = p.ngpown * pl.n_ig_tiles;
    int64_t grid = static_cast<int64_t>(sms) * bps;
    if (grid > pl.ntiles) grid = pl.ntiles;
    if (grid < 1) grid = 1;
    pl.grid = static_cast<int>(grid);
    pl.off_desc = off;
    off = gpp::align_up(off + sizeof(gpp::BatchInst));
    pl.off_counter = off;
    off = gpp::align_up(off + sizeof(unsigned long long));
    pl.off_partials = off;
    off = gpp::align_up(off + static_cast<size_t>(pl.ntiles) * 4 * p.nw * sizeof(double));
  }
  pl.total = off;
  *plan = pl;
  return GPP_OK;
}

// The descriptor of a single instance whose gather segments start at `ws`.
// The scale of achtemp and the squared cutoff factor the kernels apply (gpp_physics).
double ach_scale(const gpp_options& o) { return (o.physics & GPP_PHYS_CH_HALF) ? 0.5 : 1.0; }
double sexcut2(const gpp_options& o) {
  return (o.physics & GPP_PHYS_SX_CUTOFF) ? o.sexcut * o.sexcut : 0.0;
}

gpp::BatchInst describe(const gpp_problem& p, const gpp_options& o, bool f32,
                        const gpp::FwdPlan& pl, char* ws) {
  const int occ_mode = o.occ_mode;
  gpp::BatchInst d;
  d.B = static_cast<int>(p.number_bands);
  d.nocc = static_cast<int>(occ_mode == GPP_OCC_OCCUPIED ? std::min(p.nvband, p.number_bands)
                                                         : p.number_bands);
  d.G = p.ncouls;
  d.P = p.ngpown;
  d.n_ig_tiles = pl.n_ig_tiles;
  d.aqsn = reinterpret_cast<const double2*>(p.aqsntemp);
  d.aqsn32 = !f32            ? nullptr
             : pl.convert_c64 ? reinterpret_cast<const float2*>(ws + pl.off_aqsn32)
                              : reinterpret_cast<const float2*>(p.aqsntemp_c64);
  d.eps = reinterpret_cast<const double2*>(p.I_eps_array);
  d.wt = reinterpret_cast<const double2*>(p.wtilde_array);
  d.am = reinterpret_cast<const double2*>(ws + pl.off_am);
  d.am32 = f32 ? reinterpret_cast<const float2*>(ws + pl.off_am32) : nullptr;
  d.bt = reinterpret_cast<const gpp::BandEntry*>(ws + pl.off_bt);
  d.bt32 = f32 ? reinterpret_cast<const float4*>(ws + pl.off_bt32) : nullptr;
  d.colg = reinterpret_cast<const int*>(ws + pl.off_colvalid);
  d.flags = reinterpret_cast<const int*>(ws + pl.off_flags);
  d.ach = p.achtemp;
  d.asx = p.asxtemp;
  d.ach_scale = ach_scale(o);
  d.sx2 = sexcut2(o);
  return d;
}

int validate(const gpp_problem* prob, const gpp_options* opt, gpp_options* o);

// Adjoint workspace: the gather segments of the forward layout (with a one-CTA partial
// area), then the adjoint's band table, batch partials and per-(band, column) totals.
constexpr size_t kBwdPartialBudget = size_t(1) << 30;  // bytes for the per-batch partials

int make_bwd_plan(const gpp_problem& p, const gpp_options& o, gpp::BwdPlan* plan) {
  gpp::BwdPlan bp;
  gpp_options fo = o;
  fo.precision = GPP_FP64;
  int rc = make_plan(p, fo, &bp.fwd, true);
  if (rc) return rc;
  if (degenerate(p)) {
    *plan = bp;
    return GPP_OK;
  }
  int dev = 0, sms = 0;
  cudaError_t e = checked(cudaGetDevice(&dev));
  if (e == cudaSuccess) e = checked(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (e != cudaSuccess) return cuda_fail(e, "querying the device");
  const int bps = gpp::bwd_blocks_per_sm(static_cast<int>(p.nw));
  if (bps <= 0) return fail(GPP_ERR_CUDA, "occupancy query failed for the adjoint kernel");
  bp.max_grid = sms * bps;
  const int64_t groups = gpp::bwd_groups(p.ngpown);
  const size_t per_group = static_cast<size_t>(p.number_bands) * p.ncouls * 16;
  int64_t bg = static_cast<int64_t>(kBwdPartialBudget / (per_group ? per_group : 1));
  if (bg < 1) bg = 1;
  if (bg > groups) bg = groups;
  bp.batch_groups = static_cast<int>(bg);
  const int64_t n_ig_tiles = (p.ncouls + gpp::bwd_tile_ig() - 1) / gpp::bwd_tile_ig();
  size_t off = bp.fwd.total;
  bp.off_bwd_bt = off;
  off = gpp::align_up(off + static_cast<size_t>(p.number_bands) * p.nw * 128);
  bp.off_part_n = off;
  off = gpp::align_up(off + static_cast<size_t>(bg) * per_group);
  bp.off_part_r = off;
  off = gpp::align_up(off + static_cast<size_t>(n_ig_tiles) * p.number_bands * bg *
                                gpp::bwd_tile_cols() * 16);
  bp.off_rtot = off;
  off = gpp::align_up(off + static_cast<size_t>(p.number_bands) * p.ngpown * 16);
  bp.total = off;
  *plan = bp;
  return GPP_OK;
}

int validate(const gpp_problem* prob, const gpp_options* opt, gpp_options* o) {
  if (!prob) return fail(GPP_ERR_NULL_PTR, "problem is NULL");
  *o = opt ? *opt : defaults();
  int rc = check_options(*o);
  if (rc) return rc;
  return check_sizes(*prob);
}

}  // namespace

namespace gpp {
cudaError_t checked(cudaError_t e) {
  if (g_inject_countdown > 0 && --g_inject_countdown == 0 && e == cudaSuccess) {
    g_injected = true;
    return cudaErrorUnknown;
  }
  return e;
}

int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
void clear_error() { g_last_error.clear(); }

int sigma_workspace_query(const gpp_problem* prob, const gpp_options* opt, size_t* bytes) {
  *bytes = 0;
  gpp_options o;
  int rc = validate(prob, opt, &o);
  if (rc) return rc;
  gpp::FwdPlan plan;
  if ((rc = make_plan(*prob, o, &plan))) return rc;
  *bytes = plan.total;
  return GPP_OK;
}
}  // namespace gpp

extern "C" {

void gpp_options_default(gpp_options* opt) {
  if (opt) *opt = defaults();
}

const char* gpp_last_error(void) { return g_last_error.c_str(); }

int gpp_convert_c64(const gpp_c128* src, gpp_c64* dst, int64_t n, void* stream) {
  if (n < 0) return fail(GPP_ERR_BAD_SIZE, "n %lld is negative", (long long)n);
  if (n == 0) {
    g_last_error.clear();
    return GPP_OK;
  }
  if (!src || !dst) return fail(GPP_ERR_NULL_PTR, "src and dst must be non-NULL");
  if (!aligned(src, 16) || !aligned(dst, 8))
    return fail(GPP_ERR_NULL_PTR, "src must be 16-byte and dst 8-byte aligned");
  cudaError_t e = checked(gpp::launch_convert_c64(src, n, dst, n, 1, 0, n, static_cast<cudaStream_t>(stream)));
  if (e != cudaSuccess) return cuda_fail(e, "launching the complex64 conversion");
  g_last_error.clear();
  return GPP_OK;
}

void gpp_diag_inject_cuda_failure(int n) {
  g_inject_countdown = n > 0 ? n : 0;
  g_injected = false;
}

const char* gpp_version(void) { return "libgpp 0.1 (sm_103a)"; }

size_t gpp_sigma_workspace_size(const gpp_problem* prob, const gpp_options* opt) {
  gpp_options o;
  if (validate(prob, opt, &o)) return 0;
  gpp::FwdPlan plan;
  if (make_plan(*prob, o, &plan)) return 0;
  g_last_error.clear();
  return plan.total;
}

int gpp_sigma(const gpp_problem* prob, const gpp_options* opt, void* workspace,
              size_t workspace_bytes, void* stream) {
  gpp_options o;
  int rc = validate(prob, opt, &o);
  if (rc) return rc;
  const gpp_problem& p = *prob;
  if ((rc = check_pointers(p, o.precision))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (degenerate(p)) {
    cudaError_t e = checked(cudaMemsetAsync(p.achtemp, 0, p.nw * sizeof(gpp_c128), s));
    if (e == cudaSuccess) e = checked(cudaMemsetAsync(p.asxtemp, 0, p.nw * sizeof(gpp_c128), s));
    if (e != cudaSuccess) return cuda_fail(e, "zeroing the outputs");
    g_last_error.clear();
    return GPP_OK;
  }
  gpp::FwdPlan plan;
  if ((rc = make_plan(p, o, &plan))) return rc;
  if (!workspace) return fail(GPP_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", plan.total);
  if (!aligned(workspace, gpp::kAlign)) return fail(GPP_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (workspace_bytes < plan.total)
    return fail(GPP_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, plan.total);
  char* ws = static_cast<char*>(workspace);
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  if (o.stage_events)
    for (int i = 0; i < 4; ++i) ev[i] = static_cast<cudaEvent_t>(o.stage_events[i]);
  auto mark = [&](int i) -> cudaError_t { return ev[i] ? cudaEventRecord(ev[i], s) : cudaSuccess; };
  const bool f32 = o.precision == GPP_FP32_BULK;
  gpp::BatchInst desc = describe(p, o, f32, plan, ws);
  desc.tile0 = 0;
  desc.tile_end = plan.ntiles;
  cudaError_t e = checked(mark(0));
  if (e != cudaSuccess) return cuda_fail(e, "recording stage event 0");
  e = checked(gpp::launch_prep(p, plan, ws, f32, &desc, s));
  if (e != cudaSuccess) return cuda_fail(e, "launching the column gather");
  if (o.debug_checks) {
    int flags[4];
    e = checked(cudaMemcpyAsync(flags, ws + plan.off_flags, sizeof(flags), cudaMemcpyDeviceToHost, s));
    if (e == cudaSuccess) e = checked(cudaStreamSynchronize(s));
    if (e != cudaSuccess) return cuda_fail(e, "reading the index checks");
    if (flags[1] > 0)
      return fail(GPP_ERR_BAD_INDEX, "%d inv_igp_index / indinv entries are outside [0, ncouls]",
                  flags[1]);
  }
  if ((e = checked(mark(1))) != cudaSuccess) return cuda_fail(e, "recording stage event 1");
  const gpp::BatchInst* dptr = reinterpret_cast<const gpp::BatchInst*>(ws + plan.off_desc);
  double* partials = reinterpret_cast<double*>(ws + plan.off_partials);
  e = checked(gpp::launch_batched_main(dptr, 1, plan.ntiles, plan.nw, f32, plan.grid, plan.threads,
                               plan.igpt, reinterpret_cast<unsigned long long*>(ws + plan.off_counter),
                               partials, s));
  if (e != cudaSuccess) return cuda_fail(e, "launching the main sum");
  if ((e = checked(mark(2))) != cudaSuccess) return cuda_fail(e, "recording stage event 2");
  e = checked(gpp::launch_batched_reduce(dptr, 1, plan.nw, f32, partials, s));
  if (e != cudaSuccess) return cuda_fail(e, "launching the final reduction");
  if ((e = checked(mark(3))) != cudaSuccess) return cuda_fail(e, "recording stage event 3");
  if (o.debug_checks) {
    e = checked(cudaStreamSynchronize(s));
    if (e != cudaSuccess) return cuda_fail(e, "running the sum");
  }
  g_last_error.clear();
  return GPP_OK;
}

size_t gpp_sigma_backward_workspace_size(const gpp_problem* prob, const gpp_options* opt) {
  gpp_options o;
  if (validate(prob, opt, &o)) return 0;
  gpp::BwdPlan plan;
  if (make_bwd_plan(*prob, o, &plan)) return 0;
  g_last_error.clear();
  return plan.total;
}

int gpp_sigma_backward(const gpp_problem* prob, const gpp_options* opt,
                       const gpp_c128* grad_achtemp, const gpp_c128* grad_asxtemp,
                       const gpp_grads* grads, void* workspace, size_t workspace_bytes,
                       void* stream) {
  gpp_options o;
  int rc = validate(prob, opt, &o);
  if (rc) return rc;
  if (o.precision != GPP_FP64)
    return fail(GPP_ERR_UNSUPPORTED, "the adjoint is implemented in FP64 only");
  if (!grads) return fail(GPP_ERR_NULL_PTR, "grads is NULL");
  const gpp_problem& p = *prob;
  if ((rc = check_pointers(p, GPP_FP64, false))) return rc;
  if (!grad_achtemp || !grad_asxtemp) return fail(GPP_ERR_NULL_PTR, "output cotangents are NULL");
  gpp_c128* outs[4] = {grads->wtilde_array, grads->I_eps_array, grads->aqsmtemp, grads->aqsntemp};
  for (auto* q : outs)
    if (q && !aligned(q, 16)) return fail(GPP_ERR_NULL_PTR, "gradient arrays must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (degenerate(p)) {
    const size_t pg = static_cast<size_t>(p.ngpown) * p.ncouls * 16;
    const size_t bg = static_cast<size_t>(p.number_bands) * p.ncouls * 16;
    size_t sizes[4] = {pg, pg, bg, bg};
    for (int i = 0; i < 4; ++i)
      if (outs[i] && sizes[i]) {
        cudaError_t e = checked(cudaMemsetAsync(outs[i], 0, sizes[i], s));
        if (e != cudaSuccess) return cuda_fail(e, "zeroing gradients");
      }
    g_last_error.clear();
    return GPP_OK;
  }
  gpp::BwdPlan plan;
  if ((rc = make_bwd_plan(p, o, &plan))) return rc;
  if (!workspace || !aligned(workspace, gpp::kAlign) || workspace_bytes < plan.total)
    return fail(GPP_ERR_WORKSPACE, "adjoint workspace must be 256-byte aligned with %zu bytes",
                plan.total);
  char* ws = static_cast<char*>(workspace);
  cudaError_t e = checked(gpp::launch_prep(p, plan.fwd, ws, false, nullptr, s));
  if (e != cudaSuccess) return cuda_fail(e, "launching the column gather");
  if (o.debug_checks) {
    int flags[4];
    e = checked(cudaMemcpyAsync(flags, ws + plan.fwd.off_flags, sizeof(flags), cudaMemcpyDeviceToHost, s));
    if (e == cudaSuccess) e = checked(cudaStreamSynchronize(s));
    if (e != cudaSuccess) return cuda_fail(e, "reading the index checks");
    if (flags[1] > 0)
      return fail(GPP_ERR_BAD_INDEX, "%d inv_igp_index / indinv entries are outside [0, ncouls]",
                  flags[1]);
  }
  e = checked(gpp::launch_bwd(p, o.occ_mode, ach_scale(o), sexcut2(o), plan, ws, grad_achtemp,
                      grad_asxtemp, *grads, s));
  if (e != cudaSuccess) return cuda_fail(e, "launching the adjoint kernels");
  g_last_error.clear();
  return GPP_OK;
}

// ---------------------------------------------------------------------------------------
// Batched instances

struct gpp_batched_plan {
  int n = 0, nw = 0, threads = 128, igpt = 1, grid = 1;
  bool f32 = false;
  gpp_options opt;  // the validated options (shared by every instance)
  int64_t ntiles = 0;
  char* ws = nullptr;
  size_t total = 0, off_inst = 0, off_counter = 0, off_partials = 0;
  std::vector<gpp_problem> probs;
  std::vector<gpp::FwdPlan> iplan;
  std::vector<size_t> ioff;
  std::vector<gpp::BatchInst> inst;  // in tile order
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int batched_layout(const gpp_problem* probs, int n, const gpp_options* opt, bool check_ptrs,
                   gpp_batched_plan* bp) {
  if (!probs || n < 1) return fail(GPP_ERR_BAD_SIZE, "batched call needs n >= 1 problems");
  gpp_options o;
  int rc = validate(&probs[0], opt, &o);
  if (rc) return rc;
  bp->opt = o;
  bp->n = n;
  bp->nw = static_cast<int>(probs[0].nw);
  bp->f32 = o.precision == GPP_FP32_BULK;
  bp->threads = o.block_threads ? o.block_threads : 128;
  bp->igpt = o.ig_per_thread ? o.ig_per_thread : default_igpt(o.precision);
  int dev = 0, sms = 0;
  cudaError_t e = checked(cudaGetDevice(&dev));
  if (e == cudaSuccess) e = checked(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (e == cudaSuccess) e = gpp::batched_prepare(bp->threads, bp->nw, bp->f32, bp->igpt);
  if (e != cudaSuccess) return cuda_fail(e, "querying the device");
  int bps = o.blocks_per_sm ? o.blocks_per_sm
                            : gpp::batched_blocks_per_sm(bp->threads, bp->nw, bp->f32, bp->igpt);
  if (bps <= 0) return fail(GPP_ERR_CUDA, "occupancy query failed for the batched kernel");
  bp->grid = sms * bps;
  bp->probs.assign(probs, probs + n);
  bp->iplan.resize(n);
  bp->ioff.resize(n);
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    const gpp_problem& p = probs[i];
    if ((rc = check_sizes(p))) return rc;
    if (p.nw != bp->nw) return fail(GPP_ERR_BAD_SIZE, "instance %d has nw %lld, instance 0 has %d", i, (long long)p.nw, bp->nw);
    if (degenerate(p)) return fail(GPP_ERR_BAD_SIZE, "instance %d is empty (batched instances need B, P, G >= 1)", i);
    if (check_ptrs && (rc = check_pointers(p, o.precision))) return rc;
    if ((rc = make_plan(p, o, &bp->iplan[i], true))) return rc;
    bp->ioff[i] = off;
    off = gpp::align_up(off + bp->iplan[i].total);
  }
  // tile order: instances by band count, largest first (stable)
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return probs[a].number_bands > probs[b].number_bands; });
  const int64_t per_tile_ig = static_cast<int64_t>(bp->threads) * bp->igpt;
  bp->inst.assign(n, gpp::BatchInst());
  int64_t t0 = 0;
  for (int k = 0; k < n; ++k) {
    const int i = order[k];
    const gpp_problem& p = probs[i];
    gpp::BatchInst& d = bp->inst[k];
    d.index = i;
    d.occ_mode = o.occ_mode;
    d.n_ig_tiles = (p.ncouls + per_tile_ig - 1) / per_tile_ig;
    d.P = p.ngpown;
    d.tile0 = t0;
    t0 += d.P * d.n_ig_tiles;
    d.tile_end = t0;
  }
  bp->ntiles = t0;
  bp->off_inst = off;
  off = gpp::align_up(off + static_cast<size_t>(n) * sizeof(gpp::BatchInst));
  bp->off_counter = off;
  off = gpp::align_up(off + sizeof(unsigned long long));
  bp->off_partials = off;
  off = gpp::align_up(off + static_cast<size_t>(bp->ntiles) * 4 * bp->nw * sizeof(double));
  bp->total = off;
  return GPP_OK;
}

int batched_bind(gpp_batched_plan* bp, void* workspace, size_t bytes) {
  if (!workspace || !aligned(workspace, gpp::kAlign) || bytes < bp->total)
    return fail(GPP_ERR_WORKSPACE, "batched workspace must be 256-byte aligned with %zu bytes",
                bp->total);
  bp->ws = static_cast<char*>(workspace);
  for (int k = 0; k < bp->n; ++k) {
    gpp::BatchInst& d = bp->inst[k];
    const int i = d.index;
    gpp::FwdPlan pl = bp->iplan[i];
    pl.n_ig_tiles = d.n_ig_tiles;
    gpp::BatchInst full = describe(bp->probs[i], bp->opt, bp->f32, pl, bp->ws + bp->ioff[i]);
    full.index = i;
    full.tile0 = d.tile0;
    full.tile_end = d.tile_end;
    d = full;
  }
  return GPP_OK;
}

cudaError_t batched_enqueue(gpp_batched_plan* bp, cudaStream_t s) {
  for (int i = 0; i < bp->n; ++i) {
    cudaError_t e = checked(gpp::launch_prep(bp->probs[i], bp->iplan[i], bp->ws + bp->ioff[i], bp->f32,
                                     nullptr, s));
    if (e != cudaSuccess) return e;
  }
  const auto* inst = reinterpret_cast<const gpp::BatchInst*>(bp->ws + bp->off_inst);
  double* partials = reinterpret_cast<double*>(bp->ws + bp->off_partials);
  cudaError_t e = checked(gpp::launch_batched_main(inst, bp->n, bp->ntiles, bp->nw, bp->f32, bp->grid,
                                           bp->threads, bp->igpt,
                                           reinterpret_cast<unsigned long long*>(bp->ws + bp->off_counter),
                                           partials, s));
  if (e != cudaSuccess) return e;
  return gpp::launch_batched_reduce(inst, bp->n, bp->nw, bp->f32, partials, s);
}

}  // namespace

size_t gpp_batched_workspace_size(const gpp_problem* probs, int n, const gpp_options* opt) {
  gpp_batched_plan bp;
  if (batched_layout(probs, n, opt, false, &bp)) return 0;
  g_last_error.clear();
  return bp.total;
}

int gpp_batched_plan_create(gpp_batched_plan** plan, const gpp_problem* probs, int n,
                            const gpp_options* opt, void* workspace, size_t workspace_bytes,
                            int use_graph, void* stream) {
  if (!plan) return fail(GPP_ERR_NULL_PTR, "plan is NULL");
  *plan = nullptr;
  gpp_batched_plan* bp = new gpp_batched_plan();
  int rc = batched_layout(probs, n, opt, true, bp);
  if (!rc) rc = batched_bind(bp, workspace, workspace_bytes);
  if (rc) {
    delete bp;
    return rc;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = checked(cudaMemcpyAsync(bp->ws + bp->off_inst, bp->inst.data(),
                                  bp->inst.size() * sizeof(gpp::BatchInst), cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess) e = checked(cudaStreamSynchronize(s));
  if (e != cudaSuccess) {
    delete bp;
    return cuda_fail(e, "uploading the instance descriptors");
  }
  if (use_graph) {
    // Captured on a private stream (the caller's may be the legacy default stream, which
    // cannot be captured); the graph is later launched on the caller's stream.
    cudaStream_t cs = nullptr;
    e = checked(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    // (a capture that has begun is always ended, whatever fails inside it)
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = checked(batched_enqueue(bp, cs));
      e = checked(cudaStreamEndCapture(cs, &bp->graph));
      if (e2 != cudaSuccess) e = e2;
    }
    if (cs) cudaStreamDestroy(cs);
    if (e == cudaSuccess) e = checked(cudaGraphInstantiate(&bp->exec, bp->graph, 0));
    if (e != cudaSuccess) {
      if (bp->exec) cudaGraphExecDestroy(bp->exec);
      if (bp->graph) cudaGraphDestroy(bp->graph);
      delete bp;
      return cuda_fail(e, "capturing the batched graph");
    }
  }
  *plan = bp;
  g_last_error.clear();
  return GPP_OK;
}

int gpp_batched_plan_run(gpp_batched_plan* plan, void* stream) {
  if (!plan) return fail(GPP_ERR_NULL_PTR, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = checked(plan->exec ? cudaGraphLaunch(plan->exec, s) : batched_enqueue(plan, s));
  if (e != cudaSuccess) return cuda_fail(e, "running the batch");
  g_last_error.clear();
  return GPP_OK;
}

int gpp_batched_plan_destroy(gpp_batched_plan* plan) {
  if (!plan) return GPP_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  delete plan;
  return GPP_OK;
}

int gpp_sigma_batched(const gpp_problem* probs, int n, const gpp_options* opt, void* workspace,
                      size_t workspace_bytes, void* stream) {
  gpp_batched_plan* plan = nullptr;
  int rc = gpp_batched_plan_create(&plan, probs, n, opt, workspace, workspace_bytes, 0, stream);
  if (rc) return rc;
  rc = gpp_batched_plan_run(plan, stream);
  gpp_batched_plan_destroy(plan);
  return rc;
}

// ---------------------------------------------------------------------------------------
// Host-array variant: copies in, runs gpp_sigma on device copies inside the workspace,
// copies the outputs back and synchronises.

namespace {

struct HostLayout {
  size_t off[12];
  size_t off_counters;  // one tile counter per pipelined chunk
  size_t sigma_off;
  size_t total;
};

constexpr int kHostMaxChunks = 8;

// Segment order: aqsm, aqsn, eps, wt, vcoul, inv, indinv, wx, aqsn_c64, (two unused),
// outputs (ach then asx), then the chunk counters and gpp_sigma's workspace.
void host_layout(const gpp_problem& p, int precision, size_t sigma_bytes, HostLayout* L) {
  const size_t B = p.number_bands, G = p.ncouls, P = p.ngpown, W = p.nw;
  const bool f32 = precision == GPP_FP32_BULK;
  size_t sizes[12] = {B * G * 16, B * G * 16, P * G * 16, P * G * 16, G * 8, P * 4, (G + 1) * 4,
                      B * W * 8,  f32 ? B * G * 8 : 0, 0, 0, 2 * W * 16};
  size_t off = 0;
  for (int i = 0; i < 12; ++i) {
    L->off[i] = off;
    off = gpp::align_up(off + sizes[i]);
  }
  L->off_counters = off;
  off = gpp::align_up(off + kHostMaxChunks * sizeof(unsigned long long));
  L->sigma_off = off;
  L->total = gpp::align_up(off + sigma_bytes);
}

// The problem whose plan the host path uses: in FP32-bulk the host path always holds a
// device complex64 copy of aqsntemp (segment 8), copied from the caller's or converted chunk
// by chunk on the device, so the sum itself never converts.
gpp_problem host_sum_problem(const gpp_problem& h, int precision) {
  gpp_problem q = h;
  if (precision == GPP_FP32_BULK && !q.aqsntemp_c64)
    q.aqsntemp_c64 = reinterpret_cast<const gpp_c64*>(h.aqsntemp);  // stands for segment 8
  return q;
}

// Two streams per device for the host entry point, created on first use and kept for the
// life of the process: one for the host-to-device copies, one for every other chunk of the
// main sum (so that a chunk's last wave overlaps the next chunk's first).
struct HostStreams {
  cudaStream_t copy = nullptr, compute = nullptr;
};

std::mutex g_host_streams_mu;
std::vector<HostStreams> g_host_streams;

cudaError_t host_streams(HostStreams* out) {
  int dev = 0;
  cudaError_t e = checked(cudaGetDevice(&dev));
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_host_streams_mu);
  if (static_cast<int>(g_host_streams.size()) <= dev) g_host_streams.resize(dev + 1);
  HostStreams& hs = g_host_streams[dev];
  if (!hs.copy && (e = checked(cudaStreamCreateWithFlags(&hs.copy, cudaStreamNonBlocking))) != cudaSuccess)
    return e;
  if (!hs.compute &&
      (e = checked(cudaStreamCreateWithFlags(&hs.compute, cudaStreamNonBlocking))) != cudaSuccess)
    return e;
  *out = hs;
  return cudaSuccess;
}

// Events of one host call, destroyed when it returns.
struct EventSet {
  std::vector<cudaEvent_t> ev;
  cudaError_t make(int n) {
    ev.assign(n, nullptr);
    for (auto& x : ev) {
      cudaError_t e = checked(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  ~EventSet() {
    for (auto x : ev)
      if (x) cudaEventDestroy(x);
  }
};

}  // namespace

size_t gpp_sigma_host_workspace_size(const gpp_problem* prob, const gpp_options* opt) {
  gpp_options o;
  if (validate(prob, opt, &o)) return 0;
  gpp::FwdPlan plan;
  if (make_plan(host_sum_problem(*prob, o.precision), o, &plan)) return 0;
  HostLayout L;
  host_layout(*prob, o.precision, plan.total, &L);
  g_last_error.clear();
  return L.total;
}

int gpp_sigma_host(const gpp_problem* prob, const gpp_options* opt, void* workspace,
                   size_t workspace_bytes, void* stream) {
  gpp_options o;
  int rc = validate(prob, opt, &o);
  if (rc) return rc;
  const gpp_problem& h = *prob;
  if ((rc = check_pointers(h, o.precision))) return rc;
  gpp::FwdPlan plan;
  if ((rc = make_plan(host_sum_problem(h, o.precision), o, &plan))) return rc;
  HostLayout L;
  host_layout(h, o.precision, plan.total, &L);
  if (!workspace || !aligned(workspace, gpp::kAlign) || workspace_bytes < L.total)
    return fail(GPP_ERR_WORKSPACE, "host-call workspace must be 256-byte aligned with %zu bytes",
                L.total);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t W = h.nw;
  if (degenerate(h)) {
    cudaError_t e = checked(cudaStreamSynchronize(s));
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the stream");
    memset(h.achtemp, 0, W * sizeof(gpp_c128));
    memset(h.asxtemp, 0, W * sizeof(gpp_c128));
    g_last_error.clear();
    return GPP_OK;
  }
  char* ws = static_cast<char*>(workspace);
  const size_t B = h.number_bands, G = h.ncouls, P = h.ngpown;
  const bool f32 = o.precision == GPP_FP32_BULK;
  // aqsmtemp: the column gather reads only its B x P elements at the gathered columns. When
  // the caller's array is page-locked and mapped into the device's address space, the
  // gather reads them in place (B P 16 bytes, 13 MB at the benchmark shape, instead of a
  // B G 16-byte copy that the sum would wait for); otherwise it is copied like the rest.
  const gpp_c128* aqsm_mapped = nullptr;
  {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, h.aqsmtemp) == cudaSuccess) {
      if (pa.type == cudaMemoryTypeHost && pa.devicePointer)
        aqsm_mapped = static_cast<const gpp_c128*>(pa.devicePointer);
    } else {
      cudaGetLastError();  // an unrecognised pointer: copy it
    }
  }
  gpp_problem d = h;
  d.aqsmtemp = aqsm_mapped ? aqsm_mapped : reinterpret_cast<const gpp_c128*>(ws + L.off[0]);
  d.aqsntemp = reinterpret_cast<const gpp_c128*>(ws + L.off[1]);
  d.I_eps_array = reinterpret_cast<const gpp_c128*>(ws + L.off[2]);
  d.wtilde_array = reinterpret_cast<const gpp_c128*>(ws + L.off[3]);
  d.vcoul = reinterpret_cast<const double*>(ws + L.off[4]);
  d.inv_igp_index = reinterpret_cast<const int32_t*>(ws + L.off[5]);
  d.indinv = reinterpret_cast<const int32_t*>(ws + L.off[6]);
  d.wx_array = reinterpret_cast<const double*>(ws + L.off[7]);
  d.aqsntemp_c64 = f32 ? reinterpret_cast<const gpp_c64*>(ws + L.off[8]) : nullptr;
  d.achtemp = reinterpret_cast<gpp_c128*>(ws + L.off[11]);
  d.asxtemp = d.achtemp + W;
  char* sws = ws + L.sigma_off;

  // The copies overlap the sum. Tiles run G-vector-tile-major, so the tiles of a range of
  // G-vector tiles need only those G-vectors of aqsntemp, I_eps and wtilde: the sum runs in
  // up to kHostMaxChunks such chunks, chunk k starting once its columns are on the device,
  // on two streams in turn. Every tile writes the partial slot it has in gpp_sigma and one
  // final reduction sums them in the same order, so the result equals gpp_sigma's bit for bit.
  const int64_t nigt = plan.n_ig_tiles;
  const double chunk_bytes = 128.0 * (1 << 20);
  int K = static_cast<int>(std::min<double>(kHostMaxChunks,
                                            std::max(1.0, (2.0 * P + B) * G * 16 / chunk_bytes)));
  K = static_cast<int>(std::min<int64_t>(K, nigt));
  HostStreams hs;
  cudaError_t e = checked(host_streams(&hs));
  EventSet ev;
  // [0] start, [1] common inputs copied, [2] gather done, [3 .. 3+K) chunk k copied,
  // [3+K] last chunk on the second stream done
  if (e == cudaSuccess) e = checked(ev.make(4 + K));
  if (e != cudaSuccess) return cuda_fail(e, "creating the host path's streams and events");
  const int64_t tile_ig = static_cast<int64_t>(plan.threads) * plan.igpt;
  auto h2d = [&](size_t seg, const void* src, size_t bytes) {
    return cudaMemcpyAsync(ws + L.off[seg], src, bytes, cudaMemcpyHostToDevice, hs.copy);
  };
  auto h2d_cols = [&](size_t seg, const void* src, size_t esize, size_t rows, int64_t c0,
                      int64_t c1) {
    return cudaMemcpy2DAsync(ws + L.off[seg] + c0 * esize, G * esize,
                             static_cast<const char*>(src) + c0 * esize, G * esize,
                             (c1 - c0) * esize, rows, cudaMemcpyHostToDevice, hs.copy);
  };
  // After the first copy is enqueued, an error return first waits for the work already
  // enqueued on the three streams: the copies read the caller's host arrays and write the
  // workspace, which the caller may free as soon as the call returns.
  auto drain = [&]() {
    cudaStreamSynchronize(hs.copy);
    cudaStreamSynchronize(hs.compute);
    cudaStreamSynchronize(s);
  };
  auto drain_fail = [&](cudaError_t err, const char* what) {
    drain();
    return cuda_fail(err, what);
  };
  e = checked(cudaEventRecord(ev.ev[0], s));
  if (e == cudaSuccess) e = checked(cudaStreamWaitEvent(hs.copy, ev.ev[0], 0));
  if (e == cudaSuccess) e = checked(cudaStreamWaitEvent(hs.compute, ev.ev[0], 0));
  if (e == cudaSuccess && !aqsm_mapped) e = checked(h2d(0, h.aqsmtemp, B * G * 16));
  if (e == cudaSuccess) e = checked(h2d(4, h.vcoul, G * 8));
  if (e == cudaSuccess) e = checked(h2d(5, h.inv_igp_index, P * 4));
  if (e == cudaSuccess) e = checked(h2d(6, h.indinv, (G + 1) * 4));
  if (e == cudaSuccess) e = checked(h2d(7, h.wx_array, B * W * 8));
  if (e == cudaSuccess) e = checked(cudaEventRecord(ev.ev[1], hs.copy));
  // Chunk sizes double (boundaries at nigt (2^k - 1) / (2^K - 1), each chunk at least one
  // G-vector tile): the sum starts after a small first chunk has arrived, and every later
  // chunk arrives while the ones before it are summed.
  std::vector<int64_t> igt0(K + 1);
  igt0[0] = 0;
  for (int k = 1; k <= K; ++k) {
    const int64_t geo = static_cast<int64_t>(
        std::llround(static_cast<double>(nigt) * ((1ll << k) - 1) / ((1ll << K) - 1)));
    igt0[k] = std::min<int64_t>(std::max<int64_t>(geo, igt0[k - 1] + 1), nigt - (K - k));
  }
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    const int64_t c0 = igt0[k] * tile_ig, c1 = std::min<int64_t>(igt0[k + 1] * tile_ig, G);
    e = checked(h2d_cols(1, h.aqsntemp, 16, B, c0, c1));
    if (e == cudaSuccess && f32) {
      if (h.aqsntemp_c64)
        e = checked(h2d_cols(8, h.aqsntemp_c64, 8, B, c0, c1));
      else  // converted on the device from the chunk just copied, in copy-stream order
        e = checked(gpp::launch_convert_c64(d.aqsntemp, G, const_cast<gpp_c64*>(d.aqsntemp_c64), G, B,
                                    c0, c1, hs.copy));
    }
    if (e == cudaSuccess) e = checked(h2d_cols(2, h.I_eps_array, 16, P, c0, c1));
    if (e == cudaSuccess) e = checked(h2d_cols(3, h.wtilde_array, 16, P, c0, c1));
    if (e == cudaSuccess) e = checked(cudaEventRecord(ev.ev[3 + k], hs.copy));
  }
  if (e != cudaSuccess) return drain_fail(e, "copying inputs to the device");

  cudaEvent_t stage[4] = {nullptr, nullptr, nullptr, nullptr};
  if (o.stage_events)
    for (int i = 0; i < 4; ++i) stage[i] = static_cast<cudaEvent_t>(o.stage_events[i]);
  auto mark = [&](int i) -> cudaError_t {
    return stage[i] ? cudaEventRecord(stage[i], s) : cudaSuccess;
  };
  gpp::BatchInst desc = describe(d, o, f32, plan, sws);
  desc.tile0 = 0;
  desc.tile_end = plan.ntiles;
  e = checked(cudaStreamWaitEvent(s, ev.ev[1], 0));
  if (e == cudaSuccess) e = checked(mark(0));
  if (e == cudaSuccess) e = checked(gpp::launch_prep(d, plan, sws, f32, &desc, s));
  if (e != cudaSuccess) return drain_fail(e, "launching the column gather");
  if (o.debug_checks) {
    int flags[4];
    e = checked(cudaMemcpyAsync(flags, sws + plan.off_flags, sizeof(flags), cudaMemcpyDeviceToHost, s));
    if (e == cudaSuccess) e = checked(cudaStreamSynchronize(s));
    if (e != cudaSuccess) return drain_fail(e, "reading the index checks");
    if (flags[1] > 0) {
      drain();
      return fail(GPP_ERR_BAD_INDEX, "%d inv_igp_index / indinv entries are outside [0, ncouls]",
                  flags[1]);
    }
  }
  e = checked(cudaEventRecord(ev.ev[2], s));
  if (e == cudaSuccess) e = checked(cudaStreamWaitEvent(hs.compute, ev.ev[2], 0));
  if (e == cudaSuccess) e = checked(mark(1));
  if (e != cudaSuccess) return drain_fail(e, "launching the column gather");
  const gpp::BatchInst* dptr = reinterpret_cast<const gpp::BatchInst*>(sws + plan.off_desc);
  double* partials = reinterpret_cast<double*>(sws + plan.off_partials);
  auto* counters = reinterpret_cast<unsigned long long*>(ws + L.off_counters);
  bool second_used = false;
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    cudaStream_t sk = (k & 1) ? hs.compute : s;
    const int64_t t0 = igt0[k] * static_cast<int64_t>(P), t1 = igt0[k + 1] * static_cast<int64_t>(P);
    const int grid = static_cast<int>(std::min<int64_t>(plan.grid, t1 - t0));
    e = checked(cudaStreamWaitEvent(sk, ev.ev[3 + k], 0));
    if (e == cudaSuccess)
      e = checked(gpp::launch_batched_main(dptr, 1, t1, plan.nw, f32, grid, plan.threads, plan.igpt,
                                   counters + k, partials, sk, t0));
    second_used = second_used || (k & 1);
  }
  if (e == cudaSuccess && second_used) {
    e = checked(cudaEventRecord(ev.ev[3 + K], hs.compute));
    if (e == cudaSuccess) e = checked(cudaStreamWaitEvent(s, ev.ev[3 + K], 0));
  }
  if (e == cudaSuccess) e = checked(mark(2));
  if (e != cudaSuccess) return drain_fail(e, "launching the main sum");
  e = checked(gpp::launch_batched_reduce(dptr, 1, plan.nw, f32, partials, s));
  if (e == cudaSuccess) e = checked(mark(3));
  if (e == cudaSuccess) e = checked(cudaMemcpyAsync(h.achtemp, d.achtemp, W * 16, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess) e = checked(cudaMemcpyAsync(h.asxtemp, d.asxtemp, W * 16, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess) e = checked(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return drain_fail(e, "running the sum and copying the outputs back");
  g_last_error.clear();
  return GPP_OK;
}

}  // extern "C"
