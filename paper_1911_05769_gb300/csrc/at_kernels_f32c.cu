// at_kernels_f32c.cu -- single-domain stepper for a compensated float state
// (every value a pair hi + lo of FP32 words: stencil differences and halo
// values word by word, updates by error-free two-sums; see atk::run_pe,
// PREC 2).  The extra registers take it to two CTAs per SM.
#define AT_MIN_CTAS_PER_SM 2
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_stepper_kernel_f32c(int order, int gw, bool forced, bool full)
{
    return atk::stepper_kernel<float, false, 2>(order, gw, forced, full);
}
