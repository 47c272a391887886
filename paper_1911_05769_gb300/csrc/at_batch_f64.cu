// at_batch_f64.cu -- ensemble instantiations of the persistent AT stepper for
// double state (unforced; see atk::stepper_kernel).
#define AT_MIN_CTAS_PER_SM 2
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_batch_kernel_f64(int order, int gw, bool full)
{
    return atk::stepper_kernel<double, true>(order, gw, false, full);
}
