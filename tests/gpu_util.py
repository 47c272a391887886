"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and the
oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle

TOL = {"f64": 1e-12, "f32": 1e-5}   # relative L-inf bars for FP64 / FP32 state


def rel_linf(a, b) -> float:
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


def gpu_run(u0, *, P, order, L, nu, dt, steps, dtype="f64", mode=None, seed=0, forcing=0.0, max_ctas=0,
            stages=0, delays=None, record=False, calls=None, flags=0, timeout_ns=0, test_skip_step=0,
            steps_per_pass=0, check=True):
    """Runs the CUDA solver; returns dict(u, hist, m1, m2, rec, info, rc)."""
    import torch

    from paper_1911_05769_gb300 import AT_OK, AT_REPLAY, AT_SEEDED, Solver, binding
    mode = AT_SEEDED if mode is None else mode
    N = len(u0)
    s = Solver(N, P, order, L, nu, dt, dtype=dtype, seed=seed, forcing_amp=forcing, max_ctas=max_ctas,
               stages=stages, flags=flags, timeout_ns=timeout_ns, test_skip_step=test_skip_step,
               steps_per_pass=steps_per_pass)
    s.set_state(torch.from_numpy(np.ascontiguousarray(u0)).cuda())
    calls = calls or [steps]
    assert sum(calls) == steps
    recs, done = [], 0
    for c in calls:
        d = None
        if mode == AT_REPLAY:
            d = torch.from_numpy(np.ascontiguousarray(delays[done:done + c])).cuda()
        elif record:
            d = torch.full((c, P, 2), -1, dtype=torch.int8, device="cuda")
        s.step(c, mode, d)
        if record and mode != AT_REPLAY:
            recs.append(d)
        done += c
    out = torch.empty(N, dtype=s.tdtype, device="cuda")
    rc = binding.at_state(s.h, out.data_ptr())
    if check and rc != AT_OK:
        raise AssertionError(f"at_state returned {rc}: {binding.at_last_error()}")
    res = dict(rc=rc, info=s.info())
    if rc == AT_OK:
        hist, m1, m2 = s.delay_stats()
        res.update(u=out.cpu().numpy().astype(np.float64), hist=np.array(hist), m1=m1, m2=m2)
        if recs:
            res["rec"] = np.concatenate([r.cpu().numpy() for r in recs], axis=0)
    s.close()
    return res


def oracle_run(u0, *, P, order, L, nu, dt, steps, mode, seed=0, forcing=0.0, delays=None, per_subdomain=False,
               **kw):
    """mode: 'sync' | 'seeded' | 'replay'."""
    m = {"sync": oracle.SYNC, "seeded": oracle.SEEDED, "replay": oracle.REPLAY}[mode]
    return oracle.run(np.asarray(u0, np.float64), P=P, order=order, L=L, nu=nu, dt=dt, n_steps=steps,
                      delay_mode=m, seed=seed, forcing_amp=forcing, replay=delays, per_subdomain=per_subdomain,
                      **kw)
