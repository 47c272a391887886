// at_adjoint.cu -- instantiations of the adjoint step kernel (float and
// double state, stencil order 2 and 4).
#include "at_adjoint.cuh"

// Adjoint step kernel for word size w (4 or 8) and stencil order 2|4.
__attribute__((visibility("hidden"))) void *atk_adjoint_kernel(int w, int order)
{
    if (w == 8) return order == 2 ? (void *)atk::at_adjoint_step<double, 2> : (void *)atk::at_adjoint_step<double, 4>;
    return order == 2 ? (void *)atk::at_adjoint_step<float, 2> : (void *)atk::at_adjoint_step<float, 4>;
}
