// at_kernels_f32v.cu -- single-domain stepper for float state with the
// viscous term formed and accumulated in FP64 (close to the stability limit).
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_stepper_kernel_f32v(int order, int gw, bool forced, bool full)
{
    return atk::stepper_kernel<float, false, 1>(order, gw, forced, full);
}

