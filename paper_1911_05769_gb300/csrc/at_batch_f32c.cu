// at_batch_f32c.cu -- ensemble instantiations of the persistent AT stepper for
// a compensated float state (every value a pair hi + lo of FP32 words; see
// atk::run_pe, PREC 2).  The extra registers take it to two CTAs per SM.
#define AT_MIN_CTAS_PER_SM 2
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_batch_kernel_f32c(int order, int gw, bool full)
{
    return atk::stepper_kernel<float, true, 2>(order, gw, false, full);
}
