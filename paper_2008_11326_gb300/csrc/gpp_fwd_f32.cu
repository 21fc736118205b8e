// Forward GPP sum with FP32 bulk arithmetic (not built yet).
#include "gpp_internal.h"

namespace gpp {

bool fwd_f32_available() { return false; }

int fwd_f32_blocks_per_sm(int, int) { return 0; }

cudaError_t launch_fwd_f32(const gpp_problem&, int, const FwdPlan&, char*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace gpp
