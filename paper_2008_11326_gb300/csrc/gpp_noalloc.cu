// gpp_sigma_noalloc: gpp_sigma with its scratch in a fixed device array of the library,
// for callers that cannot hand the library a workspace (see include/gpp.h).

#include <cuda_runtime.h>

#include <stdio.h>

#include <mutex>

#include "gpp.h"
#include "gpp_internal.h"

namespace {

// The scratch. In host code this symbol is only a stand-in for the device array; its device
// address comes from cudaGetSymbolAddress, looked up once per device.
static __device__ __align__(256) unsigned char g_scratch[GPP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

bool opt_default_depth(const gpp_options& o) { return o.ig_per_thread == 0; }

}  // namespace

extern "C" int gpp_sigma_noalloc(const gpp_problem* prob, const gpp_options* opt, void* stream) {
  gpp_options o;
  if (opt) {
    o = *opt;
  } else {
    gpp_options_default(&o);
  }
  size_t need = gpp_sigma_workspace_size(prob, &o);
  if (need == 0 && gpp_last_error()[0] != '\0') return GPP_ERR_BAD_SIZE;  // invalid arguments
  // With the default tile depth, the deepest tiles (8 G-vectors per thread: half the
  // per-tile partial slots) may fit where the default does not; the result is the same sum
  // up to the order of its partials.
  if (need > GPP_NOALLOC_SCRATCH_BYTES && opt_default_depth(o)) {
    gpp_options deeper = o;
    deeper.ig_per_thread = 8;
    const size_t n = gpp_sigma_workspace_size(prob, &deeper);
    if (n != 0 && n <= GPP_NOALLOC_SCRATCH_BYTES) {
      o = deeper;
      need = n;
    }
  }
  if (need > GPP_NOALLOC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "problem needs %zu bytes of scratch; gpp_sigma_noalloc holds %zu (use gpp_sigma)",
             need, static_cast<size_t>(GPP_NOALLOC_SCRATCH_BYTES));
    return gpp::report_error(GPP_ERR_WORKSPACE, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gpp::report_error(GPP_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return gpp::report_error(GPP_ERR_UNSUPPORTED, "device ordinal too large");
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_scratch);
      if (e != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        return gpp::report_error(GPP_ERR_CUDA, cudaGetErrorString(e));
      }
    }
    ptr = g_scratch_ptr[dev];
  }
  return gpp_sigma(prob, &o, ptr, GPP_NOALLOC_SCRATCH_BYTES, stream);
}
