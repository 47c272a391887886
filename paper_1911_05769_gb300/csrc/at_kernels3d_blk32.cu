// at_kernels3d_blk32.cu -- instantiations of the temporally blocked
// free-running scalar 3D stepper for 32^3 subdomains (sizes and shared-memory
// offsets known at compile time; float and double; 2, 3 or 4 levels per
// pass; equal or unequal spacing).
#include "at_kernels3d_blk.cuh"

template <typename T, bool ISO>
static void *blk32_kernel(int sb)
{
    return sb == 2 ? (void *)atk::at_stepper3d_blk<T, 2, ISO, 32>
                   : sb == 3 ? (void *)atk::at_stepper3d_blk<T, 3, ISO, 32>
                             : (void *)atk::at_stepper3d_blk<T, 4, ISO, 32>;
}

__attribute__((visibility("hidden"))) void *atk_stepper3d_blk32_kernel(int w, int sb, int iso)
{
    if (w == 8) return iso ? blk32_kernel<double, true>(sb) : blk32_kernel<double, false>(sb);
    return iso ? blk32_kernel<float, true>(sb) : blk32_kernel<float, false>(sb);
}
