// at_kernels3d_iso.cu -- instantiations of the scalar 3D stepper for equal
// spacing on the three axes (the shapes of at_kernels3d.cu).
#include "at_kernels3d.cuh"

__attribute__((visibility("hidden"))) void *atk_stepper3d_iso_kernel(int w, int tc, int vw)
{
    if (w == 8) {
        return tc == 1 ? (void *)atk::at_stepper3d<double, 1, 1, false, 1, atk::kThreads3, true>
                       : tc == 2 ? (void *)atk::at_stepper3d<double, 2, 1, false, 1, atk::kThreads3, true>
                                 : (void *)atk::at_stepper3d<double, 4, 1, false, 1, atk::kThreads3, true>;
    }
    if (vw == 4) return (void *)atk::at_stepper3d<float, 2, 1, false, 4, 128, true>;   // 128 threads, 2 groups each
    return tc == 1 ? (void *)atk::at_stepper3d<float, 1, 1, false, 1, atk::kThreads3, true>
                   : tc == 2 ? (void *)atk::at_stepper3d<float, 2, 1, false, 1, atk::kThreads3, true>
                             : (void *)atk::at_stepper3d<float, 4, 1, false, 1, atk::kThreads3, true>;
}
