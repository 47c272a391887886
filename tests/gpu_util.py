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

    from paper_1911_05769_gb300 import AT_FLAG_COMPENSATED, AT_OK, AT_REPLAY, AT_SEEDED, Solver, binding
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
        if flags & AT_FLAG_COMPENSATED:
            res["lo"] = s.state_error().cpu().numpy().astype(np.float64)
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


def gpu_ensemble_run(instances, *, M, order, steps, dtype="f64", mode=None, record=False, calls=None,
                     max_ctas=0, stages=0, steps_per_pass=0, delays=None, tune=0, flags=0, tile_subdomains=0,
                     modes=None):
    """Runs an ensemble through the C ABI (at_create_batch); returns dict(u, hist, rec, info, solver)."""
    import torch

    import at_workloads as W
    from paper_1911_05769_gb300 import AT_FLAG_COMPENSATED, AT_FREE, AT_OK, AT_REPLAY, AT_SEEDED, EnsembleSolver, binding
    mode = AT_SEEDED if mode is None else mode
    s = EnsembleSolver(instances, M, order, dtype=dtype, max_ctas=max_ctas, stages=stages,
                       steps_per_pass=steps_per_pass, flags=flags, tile_subdomains=tile_subdomains)
    u0 = torch.from_numpy(W.ensemble_field(instances)).cuda()
    res = {}
    if tune:
        s.set_state(u0)
        res["tune"] = s.tune(tune, AT_FREE if mode == AT_REPLAY else mode)
    s.set_state(u0)
    calls = calls or [steps]
    assert sum(calls) == steps
    modes = modes or [mode] * len(calls)      # a mode per call (delays recorded in every call)
    recs, done = [], 0
    for c, md in zip(calls, modes):
        d = None
        if md == AT_REPLAY:
            d = torch.from_numpy(np.ascontiguousarray(delays[done:done + c])).cuda()
        elif record:
            d = torch.full((c, s.P, 2), -1, dtype=torch.int8, device="cuda")
        s.step(c, md, d)
        if record:
            recs.append(d)
        done += c
    out = torch.empty(s.N, dtype=s.tdtype, device="cuda")
    rc = binding.at_state(s.h, out.data_ptr())
    if rc != AT_OK:
        raise AssertionError(f"at_state returned {rc}: {binding.at_last_error()}")
    hist, m1, m2 = s.delay_stats()
    res.update(u=out.cpu().numpy().astype(np.float64), hist=np.array(hist), info=s.info(), offsets=s.offsets)
    if flags & AT_FLAG_COMPENSATED:
        # the value carried: hi + lo
        res["lo"] = s.state_error().cpu().numpy().astype(np.float64)
    if recs:
        res["rec"] = np.concatenate([r.cpu().numpy() for r in recs], axis=0)
    s.close()
    return res


def oracle_ensemble(instances, *, M, order, steps, mode, delays=None, which=None):
    """The oracle run of each instance (its own domain, delays and seed):
    returns {j: (u, hist)} for the instances in ``which`` (all by default).
    ``delays`` ([steps][P][2] over the whole ensemble) serves mode 'replay'."""
    import at_workloads as W
    m = {"sync": oracle.SYNC, "seeded": oracle.SEEDED, "replay": oracle.REPLAY}[mode]
    out, p0 = {}, 0
    for j, d in enumerate(instances):
        Pj = d["n"] // M
        if which is None or j in which:
            rep = None
            if m == oracle.REPLAY:
                rep = np.ascontiguousarray(delays[:, p0:p0 + Pj, :])
            bc = d.get("bc", 1)
            out[j] = oracle.run(W.instance_field(d), N=d["n"], P=Pj, order=order, L=d["L"], nu=d["nu"],
                                dt=d["dt"], n_steps=steps, x0=d["origin"], dx=d["length"] / d["n"],
                                bc=oracle.BC_TANH if bc == 1 else oracle.BC_PERIODIC,
                                tanh=(d["tanh_a"], d["tanh_c"], d["tanh_xc"]), delay_mode=m, seed=d["seed"],
                                replay=rep)
        p0 += Pj
    return out
