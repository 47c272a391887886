// at_sync_f32v.cu -- the blocked synchronous mode (see at_sync_f32.cu) of the
// float-state stepper with the viscous term formed and accumulated in FP64.
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_sync_kernel_f32v(int order, int gw, bool forced, bool full)
{
    return atk::stepper_kernel<float, false, 1, true>(order, gw, forced, full);
}
