// at_kernels3d.cu -- instantiations of the scalar 3D stepper (float and double
// state; 1, 2 or 4 columns per thread, or for float two groups of 4
// consecutive columns in 128-thread CTAs; unequal spacing on the axes, the
// equal-spacing instances are in at_kernels3d_iso.cu) and the 3D init kernel.
#include "at_kernels3d.cuh"

// Scalar 3D stepper for word size w (4 or 8), tc column groups per thread
// (1, 2 or 4) of vw columns (1; float also 4: 128-thread CTAs, 2 groups per thread).
__attribute__((visibility("hidden"))) void *atk_stepper3d_kernel(int w, int tc, int vw)
{
    if (w == 8) {
        return tc == 1 ? (void *)atk::at_stepper3d<double, 1, 1, false, 1>
                       : tc == 2 ? (void *)atk::at_stepper3d<double, 2, 1, false, 1>
                                 : (void *)atk::at_stepper3d<double, 4, 1, false, 1>;
    }
    if (vw == 4) return (void *)atk::at_stepper3d<float, 2, 1, false, 4, 128>;   // 128 threads, 2 groups each
    return tc == 1 ? (void *)atk::at_stepper3d<float, 1, 1, false, 1>
                   : tc == 2 ? (void *)atk::at_stepper3d<float, 2, 1, false, 1>
                             : (void *)atk::at_stepper3d<float, 4, 1, false, 1>;
}

__attribute__((visibility("hidden"))) void *atk_init3d_kernel(int w)
{
    return w == 8 ? (void *)atk::at_init3d<double> : (void *)atk::at_init3d<float>;
}
