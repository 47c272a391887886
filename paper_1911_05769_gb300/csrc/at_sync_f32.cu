// at_sync_f32.cu -- the blocked synchronous mode (AT_SYNC in passes of more
// than one level, ghost cells from edge strips; see atk::run_pe, BS) of the
// single-domain stepper for float state: its own instantiations, so that the
// other modes' kernels carry none of its code.
#include "at_kernels.cuh"

__attribute__((visibility("hidden"))) void *atk_sync_kernel_f32(int order, int gw, bool forced, bool full)
{
    return atk::stepper_kernel<float, false, 0, true>(order, gw, forced, full);
}
