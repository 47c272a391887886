"""The adjoint kernel with checkpointed recomputation (at_step_checkpointed +
at_adjoint, and the autograd Function over them) against the oracle's
discrete adjoint, element by element, and against finite differences of the
GPU forward run on the full-size adjoint workload."""
import numpy as np
import pytest

import at_workloads as W
import oracle
from gpu_util import TOL, rel_linf

pytestmark = pytest.mark.gpu


def problem(N=512, P=16, order=2, L=2, nu=0.05, steps=60, seed=5):
    x, dx = W.grid(N)
    u0 = np.sin(x) + 0.5 * np.sin(3 * x + 1)
    dt = W.dt_rule(u0, dx, nu)
    rng = np.random.default_rng(seed)
    lam_T = rng.standard_normal(N)
    return dict(N=N, P=P, order=order, L=L, nu=nu, dt=dt, steps=steps, seed=seed, u0=u0, lam_T=lam_T)


def gpu_adjoint(pr, *, mode, interval, dtype="f64", delays=None, max_ctas=0, spp=0):
    import torch

    from paper_1911_05769_gb300 import AT_FREE, AT_OK, AT_REPLAY, Solver, binding as B
    tdt = torch.float64 if dtype == "f64" else torch.float32
    s = Solver(pr["N"], pr["P"], pr["order"], pr["L"], pr["nu"], pr["dt"], dtype=dtype, seed=pr["seed"],
               max_ctas=max_ctas, steps_per_pass=spp)
    s.set_state(torch.from_numpy(pr["u0"]).cuda())
    n = pr["steps"]
    ckpt = torch.empty(B.at_checkpoint_bytes(s.h, n, interval), dtype=torch.uint8, device="cuda")
    d = None
    if mode == AT_REPLAY:
        d = torch.from_numpy(np.ascontiguousarray(delays)).cuda()
    elif mode == AT_FREE:
        d = torch.full((n, pr["P"], 2), -1, dtype=torch.int8, device="cuda")
    assert B.at_step_checkpointed(s.h, n, mode, d.data_ptr() if d is not None else None, interval,
                                  ckpt.data_ptr()) == AT_OK, B.at_last_error()
    uT = s.state().double().cpu().numpy()
    lam = torch.from_numpy(pr["lam_T"]).to(tdt).cuda()
    nb = B.at_adjoint_workspace_bytes(s.h, interval)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    amode = AT_REPLAY if mode == AT_FREE else mode
    rc, dnu = B.at_adjoint(s.h, n, amode, d.data_ptr() if d is not None else None, interval, ckpt.data_ptr(),
                           ws.data_ptr(), nb, lam.data_ptr())
    assert rc == AT_OK, B.at_last_error()
    rec = d.cpu().numpy() if d is not None else None
    s.close()
    return uT, lam.double().cpu().numpy(), dnu, rec


def oracle_adjoint(pr, *, mode, delays=None):
    return oracle.adjoint(pr["u0"], pr["lam_T"], P=pr["P"], order=pr["order"], L=pr["L"], nu=pr["nu"],
                          dt=pr["dt"], n_steps=pr["steps"], delay_mode=mode, seed=pr["seed"], replay=delays)


CASES = [
    # (order, L, mode, interval, max_ctas)
    (2, 2, "seeded", 1000, 0),
    (2, 2, "seeded", 7, 2),
    (2, 2, "seeded", 3, 0),          # interval shorter than the L + s levels a checkpoint keeps
    (4, 3, "seeded", 25, 2),
    (4, 3, "seeded", 1, 0),
    (2, 2, "sync", 20, 0),
    (4, 2, "sync", 13, 3),
    (2, 0, "seeded", 10, 0),
]


@pytest.mark.parametrize("order,L,mode,interval,max_ctas", CASES)
def test_adjoint_matches_oracle_fp64(order, L, mode, interval, max_ctas):
    from paper_1911_05769_gb300 import AT_SEEDED, AT_SYNC
    pr = problem(order=order, L=L)
    m = {"seeded": AT_SEEDED, "sync": AT_SYNC}[mode]
    uT, lam0, dnu, _ = gpu_adjoint(pr, mode=m, interval=interval, max_ctas=max_ctas)
    ouT, olam0, odnu = oracle_adjoint(pr, mode={"seeded": oracle.SEEDED, "sync": oracle.SYNC}[mode])
    assert rel_linf(uT, ouT) <= TOL["f64"]
    assert rel_linf(lam0, olam0) <= TOL["f64"]
    assert abs(dnu - odnu) <= TOL["f64"] * abs(odnu)


@pytest.mark.parametrize("order,M", [(4, 516), (2, 1020)])
def test_adjoint_long_subdomains(order, M):
    """Subdomains of 516 and 1020 points: a thread of the adjoint step takes
    several points of one subdomain (256 apart), the last ones partly idle."""
    from paper_1911_05769_gb300 import AT_SEEDED
    pr = problem(N=6 * M, P=6, order=order, L=2, steps=40, nu=0.02)
    uT, lam0, dnu, _ = gpu_adjoint(pr, mode=AT_SEEDED, interval=9)
    ouT, olam0, odnu = oracle_adjoint(pr, mode=oracle.SEEDED)
    assert rel_linf(uT, ouT) <= TOL["f64"]
    assert rel_linf(lam0, olam0) <= TOL["f64"]
    # dJ/dnu sums N * steps (~1e5) terms of both signs, in another order on
    # each side (per block on the GPU): the FP64 bound K eps sum|t| allows
    # ~1e-11 of sum|t|, a few times |dJ/dnu| here
    assert abs(dnu - odnu) <= 1e-10 * abs(odnu)


def test_adjoint_of_replayed_and_free_runs():
    from paper_1911_05769_gb300 import AT_FREE, AT_REPLAY
    pr = problem(N=640, P=20, order=2, L=3, steps=80)
    delays = W.random_delays(pr["steps"], pr["P"], pr["L"], seed=9)
    uT, lam0, dnu, _ = gpu_adjoint(pr, mode=AT_REPLAY, interval=11, delays=delays)
    ouT, olam0, odnu = oracle_adjoint(pr, mode=oracle.REPLAY, delays=delays)
    assert rel_linf(lam0, olam0) <= TOL["f64"] and abs(dnu - odnu) <= TOL["f64"] * abs(odnu)
    # free-running forward (passes of L+1 levels in the last interval): the
    # recorded delays are replayed by the adjoint and by the oracle
    uT, lam0, dnu, rec = gpu_adjoint(pr, mode=AT_FREE, interval=30, max_ctas=2, spp=pr["L"] + 1)
    assert rec.min() >= 0 and rec.max() <= pr["L"]
    ouT, olam0, odnu = oracle_adjoint(pr, mode=oracle.REPLAY, delays=rec)
    assert rel_linf(uT, ouT) <= TOL["f64"]
    assert rel_linf(lam0, olam0) <= TOL["f64"] and abs(dnu - odnu) <= TOL["f64"] * abs(odnu)


def test_adjoint_fp32_against_fp64_oracle():
    from paper_1911_05769_gb300 import AT_SEEDED
    pr = problem(order=2, L=2, steps=60)
    uT, lam0, dnu, _ = gpu_adjoint(pr, mode=AT_SEEDED, interval=16, dtype="f32")
    ouT, olam0, odnu = oracle_adjoint(pr, mode=oracle.SEEDED)
    assert rel_linf(uT, ouT) <= TOL["f32"]
    assert rel_linf(lam0, olam0) <= 1e-5
    assert abs(dnu - odnu) <= 1e-4 * abs(odnu)


def test_autograd_function_gradients():
    """at_run under torch.autograd: the gradient of ||u(T) - u_target||^2 with
    respect to u0 and nu equals the oracle's adjoint of the same run."""
    import torch

    from paper_1911_05769_gb300 import AT_SEEDED, at_run
    pr = problem(N=768, P=24, order=4, L=2, steps=50)
    target = torch.from_numpy(np.cos(W.grid(pr["N"])[0])).cuda()
    u0 = torch.from_numpy(pr["u0"]).cuda().requires_grad_(True)
    nu = torch.tensor(pr["nu"], dtype=torch.float64, device="cuda", requires_grad=True)
    uT = at_run(u0, nu, P=pr["P"], order=pr["order"], L=pr["L"], dt=pr["dt"], n_steps=pr["steps"], mode=AT_SEEDED,
                seed=pr["seed"], interval=9)
    loss = ((uT - target) ** 2).sum()
    gu0, gnu = torch.autograd.grad(loss, (u0, nu))
    lam_T = 2.0 * (uT.detach() - target).cpu().numpy()
    ouT, olam0, odnu = oracle.adjoint(pr["u0"], lam_T, P=pr["P"], order=pr["order"], L=pr["L"], nu=pr["nu"],
                                      dt=pr["dt"], n_steps=pr["steps"], delay_mode=oracle.SEEDED, seed=pr["seed"])
    assert rel_linf(uT.detach().cpu().numpy(), ouT) <= TOL["f64"]
    assert rel_linf(gu0.cpu().numpy(), olam0) <= TOL["f64"]
    assert abs(float(gnu) - odnu) <= TOL["f64"] * abs(odnu)


def _workload_loss_fn():
    """J(u0, nu) = ||u(T) - u_target||^2 of the adjoint workload on the GPU
    (FP64 forward runs), and the target."""
    import torch

    from paper_1911_05769_gb300 import AT_SEEDED, Solver
    wl = W.adjoint_workload()

    def run(u0, nu, dtype="f64"):
        s = Solver(wl["N"], wl["P"], wl["order"], wl["L"], nu, wl["dt"], dtype=dtype, seed=wl["seed"])
        s.set_state(torch.as_tensor(u0).cuda())
        s.step(wl["n_steps"], AT_SEEDED)
        out = s.state().double()
        s.close()
        return out

    target = run(wl["u0_target"], wl["nu_target"])
    return wl, run, target


def _workload_gradient(dtype, run, target, wl):
    import torch

    from paper_1911_05769_gb300 import AT_SEEDED, at_run
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u0 = torch.from_numpy(wl["u0"]).to(tdt).cuda().requires_grad_(True)
    nu = torch.tensor(wl["nu"], dtype=torch.float64, device="cuda", requires_grad=True)
    uT = at_run(u0, nu, P=wl["P"], order=wl["order"], L=wl["L"], dt=wl["dt"], n_steps=wl["n_steps"],
                mode=AT_SEEDED, seed=wl["seed"], interval=wl["interval"])
    loss = ((uT.double() - target) ** 2).sum()
    gu0, gnu = torch.autograd.grad(loss, (u0, nu))
    return gu0.double(), float(gnu)


def test_adjoint_workload_against_finite_differences():
    """N = 2^20, nu = 0.01, order 2, L = 2, seeded, 2000 steps, checkpoints
    every 100, FP64: the adjoint gradient (autograd) against central
    differences of the forward run on 16 random directions in u0, and in nu.
    J is close to quadratic in u0 and nu over these 2000 short steps, so
    central differences with steps of 1e-4 (u0) and 1 % of nu are accurate
    far below the bar."""
    import torch
    wl, run, target = _workload_loss_fn()
    gu0, gnu = _workload_gradient("f64", run, target, wl)

    def J(u, n):
        return float(((run(u, n) - target) ** 2).sum())

    rng = np.random.default_rng(16)
    base = torch.from_numpy(wl["u0"]).cuda()
    for _ in range(16):
        d = torch.from_numpy(rng.standard_normal(wl["N"])).cuda()
        eps = 1e-4
        fd = (J(base + eps * d, wl["nu"]) - J(base - eps * d, wl["nu"])) / (2 * eps)
        ad = float((gu0 * d).sum())
        assert abs(fd - ad) <= 1e-7 * abs(fd), (fd, ad)
    enu = 1e-2 * wl["nu"]
    fdnu = (J(base, wl["nu"] + enu) - J(base, wl["nu"] - enu)) / (2 * enu)
    assert abs(fdnu - gnu) <= 1e-6 * abs(fdnu), (fdnu, gnu)


def test_adjoint_workload_fp32_against_fp64():
    """The same gradient with FP32 state.  Here dt ~ 3.6e-10 and an update is
    a few hundredths of an FP32 ulp of u, so the FP32 state stays at u0 while
    the FP64 state moves by ~7e-6: the loss gradient 2 (u(T) - u_target), with
    u(T) - u_target ~ 0.01, differs at the 1e-3 level.  Bar: 1e-2 relative in
    the L2 norm of dJ/du0 and in dJ/dnu."""
    wl, run, target = _workload_loss_fn()
    g64, n64 = _workload_gradient("f64", run, target, wl)
    g32, n32 = _workload_gradient("f32", run, target, wl)
    err = float((g32 - g64).norm() / g64.norm())
    assert err <= 1e-2, err
    assert abs(n32 - n64) <= 1e-2 * abs(n64), (n32, n64)
