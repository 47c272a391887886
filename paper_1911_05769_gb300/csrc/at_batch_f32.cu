// at_batch_f32.cu -- ensemble instantiations of the persistent AT stepper for
// float state (unforced; see atk::stepper_kernel).
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_batch_kernel_f32(int order, int gw, bool full)
{
    return atk::stepper_kernel<float, true>(order, gw, false, full);
}
