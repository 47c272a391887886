// at_sync_f64.cu -- the blocked synchronous mode of the single-domain and
// ensemble steppers for double state (see at_sync_f32.cu); two CTAs per SM,
// as the other FP64 kernels.
#define AT_MIN_CTAS_PER_SM 2
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_sync_kernel_f64(int order, int gw, bool forced, bool full)
{
    return atk::stepper_kernel<double, false, 0, true>(order, gw, forced, full);
}

__attribute__((visibility("hidden"))) void *atk_sync_batch_kernel_f64(int order, int gw, bool full)
{
    return atk::stepper_kernel<double, true, 0, true>(order, gw, false, full);
}
