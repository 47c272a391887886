"""GB300-native weakly-synchronous AT solver for viscous Burgers' equation.

arXiv 1911.05769: explicit forward-Euler time-marching with asynchrony-tolerant
finite differences at subdomain boundaries (Eq. AT1/AT2), subdomains as CTAs
of one persistent CUDA kernel exchanging halos through ring buffers with
progress flags (Algorithm 2), or a grid barrier every step (Algorithm 1).

The compute path is the CUDA library ``libat.so`` (C ABI in ``include/at.h``);
this package only marshals arguments to it (``binding``) and offers a small
convenience wrapper (``Solver``) that keeps the workspace in a torch tensor.
There is no CPU fallback: importing the binding fails if the library is
missing.
"""
from .binding import (AT_BC_EXACT_TANH, AT_BC_PERIODIC, AT_ERR_ARG, AT_ERR_CUDA, AT_ERR_RESIDENCY, AT_ERR_STATE,
                      AT_ERR_TIMEOUT, AT_ERR_UNSTABLE, AT_F32, AT_F64, AT_FLAG_ALLOW_UNSTABLE,
                      AT_FLAG_COMPENSATED, AT_FLAG_PER_SUBDOMAIN_DELAY, AT_FLAG_TEST_SKIP_PUBLISH, AT_FLAG_VISCOUS_FP32, AT_FLAG_VISCOUS_FP64, AT_FREE, AT_NOALLOC_SCRATCH_BYTES, AT_OK,
                      AT_REPLAY,
                      AT_SEEDED, AT_SYNC, AtError, at_batch_workspace_bytes, at_create, at_create_batch,
                      at_delay_stats, at_destroy, at_get_info, at_grid, at_info, at_instance, at_last_error,
                      at_fma_peak, at_set_state, at_state, at_state_error, at_status, at_step, at_step_noalloc, at_tune,
                      at_tune_result,
                      at_workspace_bytes, library_path, at_adjoint, at_adjoint_workspace_bytes,
                      at_checkpoint_bytes, at_set_history, at_step_checkpointed, at_step_levels,
                      at_create_system, at_moments, at_system_workspace_bytes)
from .adjoint import at_run
from .solver import EnsembleSolver, Solver, Solver3D, System3D

__all__ = [n for n in dir() if n.startswith(("AT_", "at_"))] + ["AtError", "EnsembleSolver", "Solver", "Solver3D",
                                                                   "System3D", "library_path"]
