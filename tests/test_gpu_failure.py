"""Failure detection without a GPU fault: a CTA stops releasing its progress
flags (test knob), its neighbours' bounded waits run out, the kernel latches
AT_ERR_TIMEOUT and returns, the host reads it, and the CUDA context stays
usable for the next solver."""
import numpy as np
import pytest

import at_workloads as W
from gpu_util import TOL, gpu_run, oracle_run, rel_linf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode_name", ["seeded", "free"])
def test_stalled_neighbour_times_out_and_context_survives(require_gpu, mode_name):
    import paper_1911_05769_gb300 as at
    mode = at.AT_SEEDED if mode_name == "seeded" else at.AT_FREE
    N, P, L = 16 * 256, 16, 1
    u0 = W.u0_two_modes(N)
    _, dx = W.grid(N)
    dt = W.dt_rule(u0, dx, 0.02)
    kw = dict(P=P, order=2, L=L, nu=0.02, dt=dt, steps=200)
    g = gpu_run(u0, mode=mode, seed=3, max_ctas=4, flags=at.AT_FLAG_TEST_SKIP_PUBLISH, test_skip_step=5,
                timeout_ns=20_000_000, check=False, **kw)
    assert g["rc"] == at.AT_ERR_TIMEOUT
    # a fresh solver on the same context runs normally
    g2 = gpu_run(u0, mode=at.AT_SEEDED, seed=3, max_ctas=4, **kw)
    ref, _ = oracle_run(u0, mode="seeded", seed=3, **kw)
    assert rel_linf(g2["u"], ref) <= TOL["f64"]


def test_timeout_status_is_sticky_until_reset(require_gpu):
    """The latched status is reported by every synchronising call until
    at_set_state resets it."""
    import torch

    import paper_1911_05769_gb300 as at
    N, P = 8 * 128, 8
    u0 = W.u0_two_modes(N)
    _, dx = W.grid(N)
    dt = W.dt_rule(u0, dx, 0.02)
    s = at.Solver(N, P, 2, 1, 0.02, dt, seed=1, max_ctas=2, flags=at.AT_FLAG_TEST_SKIP_PUBLISH,
                  test_skip_step=2, timeout_ns=10_000_000)
    s.set_state(torch.from_numpy(u0).cuda())
    s.step(50, at.AT_SEEDED)
    assert s.status() == at.AT_ERR_TIMEOUT
    assert "timed out" in at.at_last_error()
    assert s.status() == at.AT_ERR_TIMEOUT
    s.set_state(torch.from_numpy(u0).cuda())
    s.step(2, at.AT_SEEDED)          # within the published levels: no wait runs out
    assert s.status() == at.AT_OK
    s.close()


@pytest.mark.parametrize("mode_name,spp", [("seeded", 1), ("free", 1), ("free", 3)])
def test_stalled_neighbour_times_out_3d(require_gpu, mode_name, spp):
    """3D (one level per pass, and the blocked free-running passes): CTA 0
    stops releasing its subdomains' flags after level 4, its neighbours'
    bounded flag waits run out, the kernel latches AT_ERR_TIMEOUT and every
    CTA returns (the others see the abort word in their flag and plane
    waits); a fresh solver on the same context then runs normally."""
    import torch

    import oracle
    import paper_1911_05769_gb300 as at
    mode = at.AT_SEEDED if mode_name == "seeded" else at.AT_FREE
    n, sub, L, nu = 32, (16, 8, 8), 2, 0.1
    u0 = W.u0_spectral3d(n, seed=4, kmax=8)
    dt = W.dt_rule(u0, 2 * np.pi / n, nu, dim=3)
    s = at.Solver3D((n, n, n), sub, L, nu, dt, dtype="f64", seed=3, max_ctas=4, steps_per_pass=spp,
                    flags=at.AT_FLAG_TEST_SKIP_PUBLISH, test_skip_step=4, timeout_ns=20_000_000)
    s.set_state(torch.from_numpy(np.ascontiguousarray(u0).ravel()).cuda())
    s.step(40, mode)
    assert s.status() == at.AT_ERR_TIMEOUT
    assert "timed out" in at.at_last_error()
    s.close()
    # a fresh solver on the same context
    s = at.Solver3D((n, n, n), sub, L, nu, dt, dtype="f64", seed=3, max_ctas=4)
    s.set_state(torch.from_numpy(np.ascontiguousarray(u0).ravel()).cuda())
    s.step(10, at.AT_SEEDED)
    assert s.status() == at.AT_OK
    out = s.state().double().cpu().numpy().reshape(u0.shape)
    s.close()
    ref, _ = oracle.run3d(u0, P=(2, 4, 4), L=L, nu=nu, dt=dt, n_steps=10, delay_mode=oracle.SEEDED, seed=3)
    assert rel_linf(out, ref) <= TOL["f64"]
