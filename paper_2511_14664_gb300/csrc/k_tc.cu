// k_tc.cu -- tensor-core fused block (placeholder until the tcgen05 kernel lands).
#include "common.cuh"
#include "internal.h"

namespace qsim {
bool tc_supported(int, int) { return false; }
size_t tc_operand_bytes(int, int) { return 0; }
cudaError_t launch_tc_prepare(const double*, int, int, void*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_tc_apply(void*, int, int, const int*, const void*, int, unsigned*, cudaStream_t, const DevInfo&) {
    return cudaErrorNotSupported;
}
}  // namespace qsim
