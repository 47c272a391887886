"""Parity at the full size of the forced order-4 workload (N = 2^26 points,
P = 65536 subdomains of 1024, L = 3, forcing 0.1 sin x), in the launch
configuration the benchmark uses (default CTAs and stages).

The oracle cannot run 6.7e11 updates, so it computes sampled subdomains one
by one: a window of subdomains around the sample, wide enough that after n
steps the values of the sample subdomain do not depend on the window's ends
(information moves R points per step).  Samples include subdomain 0 (the
periodic wrap) and the first and last subdomain of a CTA."""
import math

import numpy as np
import pytest

import at_workloads as W
import oracle
from gpu_util import TOL, gpu_run, rel_linf

pytestmark = pytest.mark.gpu

CFG = W.config("burgers1d_forced_n2p26")


@pytest.fixture(scope="module")
def u0_full():
    return W.initial_field(CFG)


def _dt(u0):
    _, dx = W.grid(CFG["N"])
    return W.dt_rule(u0, dx, CFG["nu"])


def _samples(ctas):
    P = CFG["P"]
    c = ctas // 2
    lo = c * P // ctas
    hi = (c + 1) * P // ctas
    return [0, lo, hi - 1, 40001]


def _check_windows(u_gpu, u0, dt, steps, mode, dtype, samples, delays=None):
    N, P, order = CFG["N"], CFG["P"], CFG["order"]
    M, R = N // P, order // 2
    m = math.ceil(R * steps / M) + 1
    for p in samples:
        idx_p = [(p - m + i) % P for i in range(2 * m + 1)]
        u0w = np.concatenate([u0[q * M:(q + 1) * M] for q in idx_p])
        kw = dict(N=N, P=P, order=order, L=CFG["L"], nu=CFG["nu"], dt=dt, n_steps=steps,
                  forcing_amp=CFG["forcing_amp"], p_lo=idx_p[0], p_count=2 * m + 1)
        if mode == "replay":
            dw = np.ascontiguousarray(delays[:, idx_p, :])
            ref, _ = oracle.run(u0w, delay_mode=oracle.REPLAY, replay=dw, **kw)
        elif mode == "seeded":
            ref, _ = oracle.run(u0w, delay_mode=oracle.SEEDED, seed=CFG["seed"], **kw)
        else:
            ref, _ = oracle.run(u0w, delay_mode=oracle.SYNC, **kw)
        want = ref[m * M:(m + 1) * M]
        got = u_gpu[p * M:(p + 1) * M]
        scale = np.max(np.abs(u0))
        assert np.max(np.abs(got - want)) / scale <= TOL[dtype], (p, np.max(np.abs(got - want)) / scale)


def test_full_size_seeded_fp32_all_steps(require_gpu, u0_full):
    """FP32 state, seeded delays, the workload's 10^4 steps."""
    from paper_1911_05769_gb300 import AT_SEEDED
    dt = _dt(u0_full)
    steps = CFG["n_steps"]
    g = gpu_run(u0_full, P=CFG["P"], order=CFG["order"], L=CFG["L"], nu=CFG["nu"], dt=dt, steps=steps,
                dtype="f32", mode=AT_SEEDED, seed=CFG["seed"], forcing=CFG["forcing_amp"])
    assert g["hist"].sum() == steps * CFG["P"] * 2
    _check_windows(g["u"], u0_full, dt, steps, "seeded", "f32", _samples(g["info"].ctas))


def test_full_size_free_fp32_replays(require_gpu, u0_full):
    """Free-running delays at full size: record, then replay the windows."""
    from paper_1911_05769_gb300 import AT_FREE
    dt = _dt(u0_full)
    steps = 1000
    g = gpu_run(u0_full, P=CFG["P"], order=CFG["order"], L=CFG["L"], nu=CFG["nu"], dt=dt, steps=steps,
                dtype="f32", mode=AT_FREE, forcing=CFG["forcing_amp"], record=True)
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= CFG["L"]
    _check_windows(g["u"], u0_full, dt, steps, "replay", "f32", _samples(g["info"].ctas), delays=rec)


def test_full_size_blocked_free_fp32_replays(require_gpu, u0_full):
    """The benchmark's headline mode: free running with passes of L+1 levels."""
    from paper_1911_05769_gb300 import AT_FREE
    dt = _dt(u0_full)
    steps = 1000
    g = gpu_run(u0_full, P=CFG["P"], order=CFG["order"], L=CFG["L"], nu=CFG["nu"], dt=dt, steps=steps,
                dtype="f32", mode=AT_FREE, forcing=CFG["forcing_amp"], record=True, steps_per_pass=CFG["L"] + 1)
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= CFG["L"]
    _check_windows(g["u"], u0_full, dt, steps, "replay", "f32", _samples(g["info"].ctas), delays=rec)


def test_full_size_sync_fp32(require_gpu, u0_full):
    from paper_1911_05769_gb300 import AT_SYNC
    dt = _dt(u0_full)
    steps = 1000
    g = gpu_run(u0_full, P=CFG["P"], order=CFG["order"], L=CFG["L"], nu=CFG["nu"], dt=dt, steps=steps,
                dtype="f32", mode=AT_SYNC, forcing=CFG["forcing_amp"])
    _check_windows(g["u"], u0_full, dt, steps, "sync", "f32", _samples(g["info"].ctas))


def test_full_size_seeded_fp64(require_gpu, u0_full):
    from paper_1911_05769_gb300 import AT_SEEDED
    dt = _dt(u0_full)
    steps = 300
    g = gpu_run(u0_full, P=CFG["P"], order=CFG["order"], L=CFG["L"], nu=CFG["nu"], dt=dt, steps=steps,
                dtype="f64", mode=AT_SEEDED, seed=CFG["seed"], forcing=CFG["forcing_amp"])
    _check_windows(g["u"], u0_full, dt, steps, "seeded", "f64", _samples(g["info"].ctas))
