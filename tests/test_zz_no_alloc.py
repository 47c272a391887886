"""The allocation-free entry point, at_step_noalloc.

It is meant for callers that cannot allocate device memory (for instance a
plug-in whose host application owns all device memory and hands over only
the state buffer): its scratch lives in a fixed array inside the library.
These tests call it through the C ABI and check that it gives the same
result as the workspace path (at_create + at_set_state + at_step) within the
tolerance the other GPU tests use, on two calls in a row -- the second call
must not see anything the first left in the shared array -- and that a
problem too large for the array is refused with a clear message.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import math

import numpy as np
import pytest

import at_workloads as W
from gpu_util import TOL, rel_linf

pytestmark = pytest.mark.gpu


def _grid(B, N, dtype, stream, forcing, seed):
    g = B.at_grid()
    g.dim, g.bc = 1, B.AT_BC_PERIODIC
    g.dtype = B.AT_F64 if dtype == "f64" else B.AT_F32
    g.n[0], g.n[1], g.n[2] = N, 1, 1
    g.length[0] = 2 * math.pi
    g.forcing_amp = forcing
    g.seed = seed
    g.stream = stream
    return g


CALLS = [
    # N, P, order, L, dtype, forcing, seed, steps
    (64 * 256, 64, 4, 3, "f64", 0.1, 11, 300),
    (32 * 128, 32, 2, 2, "f32", 0.0, 12, 200),
]


def test_noalloc_matches_workspace_path_on_two_calls_in_a_row(require_gpu):
    import torch

    import paper_1911_05769_gb300 as at
    from paper_1911_05769_gb300 import binding as B
    stream = torch.cuda.current_stream()
    for N, P, order, L, dtype, forcing, seed, steps in CALLS:
        u0 = W.u0_fourier(N, modes=64, seed=seed)
        _, dx = W.grid(N)
        nu = 0.02
        dt = W.dt_rule(u0, dx, nu)
        tdt = torch.float64 if dtype == "f64" else torch.float32
        # the existing entry points, with a caller-allocated workspace
        s = at.Solver(N, P, order, L, nu, dt, dtype=dtype, forcing_amp=forcing, seed=seed)
        s.set_state(torch.from_numpy(u0).cuda())
        s.step(steps, at.AT_SEEDED)
        ref = s.state().cpu().numpy().astype(np.float64)
        s.close()
        # the allocation-free entry point on the caller's state buffer
        u = torch.from_numpy(u0).to(device="cuda", dtype=tdt).contiguous()
        g = _grid(B, N, dtype, stream.cuda_stream, forcing, seed)
        rc = B.at_step_noalloc(g, P, order, L, nu, dt, u.data_ptr(), steps, at.AT_SEEDED, None)
        assert rc == at.AT_OK, B.at_last_error()
        got = u.cpu().numpy().astype(np.float64)
        assert rel_linf(got, ref) <= TOL[dtype]


def test_noalloc_refuses_problems_larger_than_its_array(require_gpu):
    import torch

    import paper_1911_05769_gb300 as at
    from paper_1911_05769_gb300 import binding as B
    P = 65536                      # 65536 subdomains x 16 slots x 32 bytes > 8 MiB
    N = P * 16
    u = torch.zeros(N, dtype=torch.float32, device="cuda")
    g = _grid(B, N, "f32", torch.cuda.current_stream().cuda_stream, 0.0, 1)
    rc = B.at_step_noalloc(g, P, 4, 3, 1e-3, 1e-9, u.data_ptr(), 10, at.AT_SEEDED, None)
    assert rc == at.AT_ERR_ARG
    msg = B.at_last_error()
    assert "scratch" in msg and str(at.AT_NOALLOC_SCRATCH_BYTES) in msg
