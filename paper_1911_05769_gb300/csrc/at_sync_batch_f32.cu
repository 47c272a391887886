// at_sync_batch_f32.cu -- the blocked synchronous mode of the ensemble
// stepper for float state (see at_sync_f32.cu).
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_sync_batch_kernel_f32(int order, int gw, bool full)
{
    return atk::stepper_kernel<float, true, 0, true>(order, gw, false, full);
}
