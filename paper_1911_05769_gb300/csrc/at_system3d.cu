// at_system3d.cu -- instantiations of the 3D stepper for the system of Eq. BS
// (velocity u, v, w and 0..2 passive scalars: 3, 4 or 5 fields; float and
// double state; 1 or 2 columns per thread, or for float one group of 4
// consecutive columns).
#include "at_kernels3d.cuh"

namespace {
template <typename T, int TC, int VW, int NT = atk::kThreads3>
void *system_for(int nf)
{
    return nf == 3 ? (void *)atk::at_stepper3d<T, TC, 3, true, VW, NT>
                   : nf == 4 ? (void *)atk::at_stepper3d<T, TC, 4, true, VW, NT>
                             : (void *)atk::at_stepper3d<T, TC, 5, true, VW, NT>;
}
}  // namespace

// System stepper for word size w (4 or 8), tc column groups per thread (1 or
// 2) of vw columns (1; float also 4 with tc 1) and nf fields (3, 4 or 5).
__attribute__((visibility("hidden"))) void *atk_system3d_kernel(int w, int tc, int nf, int vw)
{
    if (w == 8) return tc == 1 ? system_for<double, 1, 1>(nf) : system_for<double, 2, 1>(nf);
    if (vw == 4) return system_for<float, 1, 4>(nf);
    return tc == 1 ? system_for<float, 1, 1>(nf) : system_for<float, 2, 1>(nf);
}
