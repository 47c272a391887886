// at_adjoint.cu -- instantiations of the adjoint interval kernel (float and
// double state, stencil order 2 and 4).
#include "at_adjoint.cuh"

// Adjoint kernel (one checkpoint interval per launch) for word size w (4 or
// 8) and stencil order 2|4.
__attribute__((visibility("hidden"))) void *atk_adjoint_kernel(int w, int order)
{
    if (w == 8) return order == 2 ? (void *)atk::at_adjoint_interval<double, 2> : (void *)atk::at_adjoint_interval<double, 4>;
    return order == 2 ? (void *)atk::at_adjoint_interval<float, 2> : (void *)atk::at_adjoint_interval<float, 4>;
}

// The one-subdomain-per-block variant (see atk::at_adjoint_own), FP32 order 2
// (where its per-thread data fits the registers; the host picks it only there).
__attribute__((visibility("hidden"))) void *atk_adjoint_own_kernel(int w, int order)
{
    (void)w;
    (void)order;
    return (void *)atk::at_adjoint_own<float, 2>;
}
