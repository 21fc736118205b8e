// gpp_sigma_noalloc: gpp_sigma with its scratch in a fixed device array of the library,
// for callers that cannot hand the library a workspace (see include/gpp.h).

#include <cuda_runtime.h>

#include <stdio.h>

#include "gpp.h"
#include "gpp_internal.h"

namespace {

// The scratch. In host code this symbol is only a stand-in for the device array; its device
// address comes from cudaGetSymbolAddress with the caller's device (and context) current.
static __device__ __align__(256) unsigned char g_scratch[GPP_NOALLOC_SCRATCH_BYTES];

}  // namespace

extern "C" int gpp_sigma_noalloc(const gpp_problem* prob, const gpp_options* opt, void* stream) {
  gpp_options o;
  if (opt) {
    o = *opt;
  } else {
    gpp_options_default(&o);
  }
  size_t need = 0;
  int rc = gpp::sigma_workspace_query(prob, &o, &need);
  if (rc != GPP_OK) return rc;  // the code gpp_sigma would return for these arguments
  // With the default tile depth, the deepest tiles (8 G-vectors per thread: half the
  // per-tile partial slots) may fit where the default does not; the result is the same sum
  // up to the order of its partials.
  if (need > GPP_NOALLOC_SCRATCH_BYTES && o.ig_per_thread == 0) {
    gpp_options deeper = o;
    deeper.ig_per_thread = 8;
    size_t n = 0;
    if (gpp::sigma_workspace_query(prob, &deeper, &n) == GPP_OK &&
        n <= GPP_NOALLOC_SCRATCH_BYTES) {
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
  // Looked up on every call rather than cached: the address belongs to the module as loaded
  // in the current context, which differs between devices and can change (another context
  // on the same device, a device reset). Once the module is loaded the lookup is a host-side
  // table query.
  void* ptr = nullptr;
  cudaError_t e = gpp::checked(cudaGetSymbolAddress(&ptr, g_scratch));
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "looking up the scratch array: %s", cudaGetErrorString(e));
    return gpp::report_error(GPP_ERR_CUDA, msg);
  }
  return gpp_sigma(prob, &o, ptr, GPP_NOALLOC_SCRATCH_BYTES, stream);
}
