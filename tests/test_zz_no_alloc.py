"""The allocation-free entry point, at_step_noalloc.

It is meant for callers that cannot allocate device memory -- for instance a
plug-in whose host application owns all device memory and hands over only
the state buffer, or code running under a hard device-memory budget: its
scratch lives in a fixed array inside the library.  These tests call it
through the C ABI and check it against the workspace path (at_create +
at_set_state + at_step) on several calls in a row, each reusing the array
the previous call left dirty:

* prescribed delays (AT_SEEDED), zero delays (AT_SYNC) and replayed delays
  (AT_REPLAY): the same kernel on the same launch shape, so the results must
  be equal bit for bit;
* free-running delays (AT_FREE, delays recorded): the oracle replaying the
  recorded delays, within the bars of the other GPU tests;

and that a problem too large for the array, or a request for temporal
blocking, is refused with a clear message.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import math

import numpy as np
import pytest

import at_workloads as W
from gpu_util import TOL, oracle_run, rel_linf

pytestmark = pytest.mark.gpu


def _grid(B, N, dtype, stream, forcing, seed, steps_per_pass=0):
    g = B.at_grid()
    g.dim, g.bc = 1, B.AT_BC_PERIODIC
    g.dtype = B.AT_F64 if dtype == "f64" else B.AT_F32
    g.n[0], g.n[1], g.n[2] = N, 1, 1
    g.length[0] = 2 * math.pi
    g.forcing_amp = forcing
    g.seed = seed
    g.stream = stream
    g.steps_per_pass = steps_per_pass
    return g


CALLS = [
    # N, P, order, L, dtype, forcing, seed, steps, mode
    (64 * 256, 64, 4, 3, "f64", 0.1, 11, 300, "seeded"),
    (32 * 128, 32, 2, 2, "f32", 0.0, 12, 200, "seeded"),
    (48 * 256, 48, 4, 3, "f32", 0.1, 13, 150, "sync"),
    (40 * 128, 40, 2, 2, "f64", 0.0, 14, 120, "replay"),
    (64 * 256, 64, 4, 3, "f32", 0.1, 15, 160, "free"),
    (32 * 128, 32, 2, 2, "f64", 0.0, 16, 200, "free"),
]


def _call(at, B, u0, N, P, order, L, nu, dt, dtype, forcing, seed, steps, mode, delays):
    import torch
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u = torch.from_numpy(u0).to(device="cuda", dtype=tdt).contiguous()
    g = _grid(B, N, dtype, torch.cuda.current_stream().cuda_stream, forcing, seed)
    m = {"seeded": at.AT_SEEDED, "sync": at.AT_SYNC, "replay": at.AT_REPLAY, "free": at.AT_FREE}[mode]
    d = None
    if mode == "replay":
        d = torch.from_numpy(delays).cuda()
    elif mode == "free":
        d = torch.full((steps, P, 2), -1, dtype=torch.int8, device="cuda")
    rc = B.at_step_noalloc(g, P, order, L, nu, dt, u.data_ptr(), steps, m, None if d is None else d.data_ptr())
    assert rc == at.AT_OK, B.at_last_error()
    rec = d.cpu().numpy() if mode == "free" else None
    return u.cpu().numpy().astype(np.float64), rec


def test_noalloc_matches_workspace_path_on_calls_in_a_row(require_gpu):
    import torch

    import paper_1911_05769_gb300 as at
    from paper_1911_05769_gb300 import binding as B
    for N, P, order, L, dtype, forcing, seed, steps, mode in CALLS:
        u0 = W.u0_fourier(N, modes=64, seed=seed)
        _, dx = W.grid(N)
        nu = 0.02
        dt = W.dt_rule(u0, dx, nu)
        delays = W.random_delays(steps, P, L, seed=seed) if mode == "replay" else None
        got, rec = _call(at, B, u0, N, P, order, L, nu, dt, dtype, forcing, seed, steps, mode, delays)
        if mode == "free":
            # any admissible delay pattern is a correct result: the oracle
            # replays the one this call recorded
            assert rec.min() >= 0 and rec.max() <= L
            ref, _ = oracle_run(u0 if dtype == "f64" else u0.astype(np.float32), P=P, order=order, L=L, nu=nu,
                                dt=dt, steps=steps, mode="replay", forcing=forcing, delays=rec)
            assert rel_linf(got, ref) <= TOL[dtype], (N, P, dtype)
            continue
        # the existing entry points, with a caller-allocated workspace
        s = at.Solver(N, P, order, L, nu, dt, dtype=dtype, forcing_amp=forcing, seed=seed)
        s.set_state(torch.from_numpy(u0).cuda())
        m = {"seeded": at.AT_SEEDED, "sync": at.AT_SYNC, "replay": at.AT_REPLAY}[mode]
        s.step(steps, m, torch.from_numpy(delays).cuda() if delays is not None else None)
        ref = s.state().cpu().numpy().astype(np.float64)
        s.close()
        assert np.array_equal(got, ref), (mode, N, P, dtype, rel_linf(got, ref))


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


def test_noalloc_refuses_temporal_blocking(require_gpu):
    import torch

    import paper_1911_05769_gb300 as at
    from paper_1911_05769_gb300 import binding as B
    N, P = 32 * 128, 32
    u = torch.zeros(N, dtype=torch.float32, device="cuda")
    g = _grid(B, N, "f32", torch.cuda.current_stream().cuda_stream, 0.0, 1, steps_per_pass=2)
    rc = B.at_step_noalloc(g, P, 2, 2, 1e-3, 1e-6, u.data_ptr(), 10, at.AT_FREE, None)
    assert rc == at.AT_ERR_ARG
    assert "steps_per_pass" in B.at_last_error()
