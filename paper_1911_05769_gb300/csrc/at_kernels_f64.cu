// at_kernels_f64.cu -- instantiations of the persistent AT stepper for double state
// (one translation unit per word size and kind, so they build in parallel).
// FP64 tiles need more registers per thread: two CTAs per SM
#define AT_MIN_CTAS_PER_SM 2
#include "at_kernels.cuh"

// Single-domain stepper kernel (see atk::stepper_kernel).
__attribute__((visibility("hidden"))) void *atk_stepper_kernel_f64(int order, int gw, bool forced, bool full)
{
    return atk::stepper_kernel<double, false>(order, gw, forced, full);
}

// State (re)initialisation kernel for stencil order 2|4.
__attribute__((visibility("hidden"))) void *atk_init_kernel_f64(int order)
{
    return order == 2 ? (void *)atk::at_init<double, 1> : (void *)atk::at_init<double, 2>;
}

// Restart kernel (stored levels -> ring, flags, level) for stencil order 2|4.
__attribute__((visibility("hidden"))) void *atk_restore_kernel_f64(int order)
{
    return order == 2 ? (void *)atk::at_restore<double, 1> : (void *)atk::at_restore<double, 2>;
}
