// at_kernels_f32.cu -- instantiations of the persistent AT stepper for float state
// (one translation unit per word size, so the two build in parallel).
#include "at_kernels.cuh"

namespace {

template <int ORDER, bool FORCED, bool FULL>
void *stepper_for(int gw)
{
    switch (gw) {
    case 1: return (void *)atk::at_stepper<float, ORDER, 1, FORCED, FULL>;
    case 2: return (void *)atk::at_stepper<float, ORDER, 2, FORCED, FULL>;
    case 4: return (void *)atk::at_stepper<float, ORDER, 4, FORCED, FULL>;
    default: return (void *)atk::at_stepper<float, ORDER, 8, FORCED, FULL>;
    }
}

template <int ORDER, bool FORCED>
void *stepper_for(int gw, bool full)
{
    return full ? stepper_for<ORDER, FORCED, true>(gw) : stepper_for<ORDER, FORCED, false>(gw);
}

}  // namespace

// Stepper kernel for stencil order 2|4, gw groups of 4 points per lane
// (1, 2, 4 or 8), with or without forcing, and full tiles (M = 128 gw) or not.
__attribute__((visibility("hidden"))) void *atk_stepper_kernel_f32(int order, int gw, bool forced, bool full)
{
    if (order == 2) return forced ? stepper_for<2, true>(gw, full) : stepper_for<2, false>(gw, full);
    return forced ? stepper_for<4, true>(gw, full) : stepper_for<4, false>(gw, full);
}

// State (re)initialisation kernel for stencil order 2|4.
__attribute__((visibility("hidden"))) void *atk_init_kernel_f32(int order)
{
    return order == 2 ? (void *)atk::at_init<float, 1> : (void *)atk::at_init<float, 2>;
}
