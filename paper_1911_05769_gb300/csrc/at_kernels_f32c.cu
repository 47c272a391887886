// at_kernels_f32c.cu -- single-domain stepper for float state with a
// compensated state (a second FP32 word per point carries the rounding error
// of the stored value; updates are error-free two-sums).  The extra registers
// take it to two CTAs per SM.
#define AT_MIN_CTAS_PER_SM 2
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_stepper_kernel_f32c(int order, int gw, bool forced, bool full)
{
    return atk::stepper_kernel<float, false, 2>(order, gw, forced, full);
}
