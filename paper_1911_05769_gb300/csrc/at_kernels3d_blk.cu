// at_kernels3d_blk.cu -- instantiations of the temporally blocked free-running
// scalar 3D stepper (float and double state; 2, 3 or 4 levels per pass;
// equal or unequal spacing on the three axes; any subdomain shape).  The
// instances for 32^3 subdomains are in at_kernels3d_blk32.cu.
#include "at_kernels3d_blk.cuh"

template <typename T, bool ISO>
static void *blk_kernel(int sb)
{
    return sb == 2 ? (void *)atk::at_stepper3d_blk<T, 2, ISO>
                   : sb == 3 ? (void *)atk::at_stepper3d_blk<T, 3, ISO> : (void *)atk::at_stepper3d_blk<T, 4, ISO>;
}

__attribute__((visibility("hidden"))) void *atk_stepper3d_blk_kernel(int w, int sb, int iso)
{
    if (w == 8) return iso ? blk_kernel<double, true>(sb) : blk_kernel<double, false>(sb);
    return iso ? blk_kernel<float, true>(sb) : blk_kernel<float, false>(sb);
}
