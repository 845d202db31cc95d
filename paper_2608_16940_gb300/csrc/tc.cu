// Split-TF32 tensor-core fused update (placeholder until the tcgen05 kernel lands).
#include "qsa_internal.h"
#include "qsa_runtime.h"

namespace qsa {
bool tc_available(qsa_state, int) { return false; }
cudaError_t launch_apply_tc(float2*, int, const int*, int, const float*, int*, cudaStream_t, uint64_t*) {
    return cudaErrorNotSupported;
}
}  // namespace qsa
