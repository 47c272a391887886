// at_kernels_f32.cu -- instantiations of the persistent AT stepper for float state
// (one translation unit per word size and kind, so they build in parallel).
#include "at_kernels.cuh"

// Single-domain stepper kernel (see atk::stepper_kernel).
__attribute__((visibility("hidden"))) void *atk_stepper_kernel_f32(int order, int gw, bool forced, bool full)
{
    return atk::stepper_kernel<float, false>(order, gw, forced, full);
}

// State (re)initialisation kernel for stencil order 2|4.
__attribute__((visibility("hidden"))) void *atk_init_kernel_f32(int order)
{
    return order == 2 ? (void *)atk::at_init<float, 1> : (void *)atk::at_init<float, 2>;
}

// Restart kernel (stored levels -> ring, flags, level) for stencil order 2|4.
__attribute__((visibility("hidden"))) void *atk_restore_kernel_f32(int order)
{
    return order == 2 ? (void *)atk::at_restore<float, 1> : (void *)atk::at_restore<float, 2>;
}
