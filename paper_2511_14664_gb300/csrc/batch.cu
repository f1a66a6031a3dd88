// batch.cu -- many independent circuits in one persistent launch (placeholder until the kernel lands).
#include "capi_state.h"
#include "internal.h"

using namespace qsim;

extern "C" {
int qsim_batch_workspace_bytes(const qsim_circuit*, int, size_t*) {
    set_error("batched execution is not built yet");
    return QSIM_EUNSUPPORTED;
}
int qsim_batch_run(const qsim_circuit*, int, const qsim_run_opts*, void*, size_t, void*, double*, double*,
                   qsim_plan_info*) {
    set_error("batched execution is not built yet");
    return QSIM_EUNSUPPORTED;
}
}
