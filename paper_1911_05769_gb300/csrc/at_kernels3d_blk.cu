// at_kernels3d_blk.cu -- instantiations of the temporally blocked free-running
// scalar 3D stepper (float and double state; 2, 3 or 4 levels per pass).
#include "at_kernels3d_blk.cuh"

__attribute__((visibility("hidden"))) void *atk_stepper3d_blk_kernel(int w, int sb)
{
    if (w == 8) {
        return sb == 2 ? (void *)atk::at_stepper3d_blk<double, 2>
                       : sb == 3 ? (void *)atk::at_stepper3d_blk<double, 3> : (void *)atk::at_stepper3d_blk<double, 4>;
    }
    return sb == 2 ? (void *)atk::at_stepper3d_blk<float, 2>
                   : sb == 3 ? (void *)atk::at_stepper3d_blk<float, 3> : (void *)atk::at_stepper3d_blk<float, 4>;
}
