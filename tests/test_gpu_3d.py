"""The 3D stepper (scalar Burgers, order 2, AT halos on six faces) against the
3D oracle, element by element, on seeded k^-5/3 fields."""
import numpy as np
import pytest

import at_workloads as W
import oracle
from gpu_util import TOL, rel_linf

pytestmark = pytest.mark.gpu


def gpu_run3d(u0, *, sub, L, nu, dt, steps, dtype="f64", mode=None, seed=0, max_ctas=0, stages=0, delays=None,
              record=False, calls=None, length=(2 * np.pi,) * 3, steps_per_pass=0):
    import torch

    from paper_1911_05769_gb300 import AT_OK, AT_REPLAY, AT_SEEDED, Solver3D, binding
    mode = AT_SEEDED if mode is None else mode
    n2, n1, n0 = u0.shape
    s = Solver3D((n0, n1, n2), sub, L, nu, dt, dtype=dtype, seed=seed, max_ctas=max_ctas, stages=stages,
                 length=length, steps_per_pass=steps_per_pass)
    s.set_state(torch.from_numpy(np.ascontiguousarray(u0).ravel()).cuda())
    calls = calls or [steps]
    recs, done = [], 0
    for c in calls:
        d = None
        if mode == AT_REPLAY:
            d = torch.from_numpy(np.ascontiguousarray(delays[done:done + c])).cuda()
        elif record:
            d = torch.full((c, s.P, 6), -1, dtype=torch.int8, device="cuda")
        s.step(c, mode, d)
        if record and mode != AT_REPLAY:
            recs.append(d)
        done += c
    out = torch.empty(s.N, dtype=s.tdtype, device="cuda")
    rc = binding.at_state(s.h, out.data_ptr())
    assert rc == AT_OK, binding.at_last_error()
    hist, _, _ = s.delay_stats()
    res = dict(u=out.double().cpu().numpy().reshape(u0.shape), hist=np.array(hist), info=s.info(), P=s.P)
    if recs:
        res["rec"] = np.concatenate([r.cpu().numpy() for r in recs], axis=0)
    s.close()
    return res


# viscosity with a cell Peclet number max|u| dx / nu of about 2 (forward Euler
# with central advection diverges far above that)
NU = {24: 0.15, 32: 0.1, 256: 0.0125}


def case(n, seed=4, kmax=8):
    u0 = W.u0_spectral3d(n, seed=seed, kmax=kmax)
    dx = 2 * np.pi / n
    return u0, W.dt_rule(u0, dx, NU[n], dim=3)


SHAPES = [
    # (n, sub, max_ctas)
    (32, (16, 16, 8), 0),
    (32, (16, 16, 8), 3),            # several subdomains per CTA, uneven split
    (32, (32, 8, 4), 5),
    (24, (8, 4, 3), 0),              # 96 subdomains of 96 points; most threads idle
    (32, (32, 32, 16), 0),           # 4 columns per thread
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,sub,max_ctas", SHAPES)
def test_seeded_3d_matches_oracle(dtype, n, sub, max_ctas):
    from paper_1911_05769_gb300 import AT_SEEDED
    u0, dt = case(n)
    nu, L, steps = NU[n], 2, 40
    P = tuple(n // m for m in sub)
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=steps, dtype=dtype, mode=AT_SEEDED, seed=5,
                  max_ctas=max_ctas)
    ref, hist = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=steps, delay_mode=oracle.SEEDED, seed=5)
    assert rel_linf(g["u"], ref) <= TOL[dtype]
    assert np.array_equal(g["hist"], hist)
    # FP32 planes of 1024 points run in 128-thread CTAs of 4-column groups
    assert g["info"].threads == (128 if dtype == "f32" and sub[0] * sub[1] == 1024 else 256)


def test_sync_replay_and_free_3d():
    from paper_1911_05769_gb300 import AT_FREE, AT_REPLAY, AT_SYNC
    n, sub, L = 32, (16, 8, 8), 3
    nu = NU[n]
    u0, dt = case(n, seed=7)
    P = tuple(n // m for m in sub)
    NP = P[0] * P[1] * P[2]
    steps = 36
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=steps, mode=AT_SYNC, max_ctas=4)
    ref, _ = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=steps, delay_mode=oracle.SYNC)
    assert rel_linf(g["u"], ref) <= TOL["f64"]
    d = np.random.default_rng(3).integers(0, L + 1, size=(steps, NP, 6), dtype=np.int8)
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=steps, mode=AT_REPLAY, delays=d)
    ref, _ = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=steps, delay_mode=oracle.REPLAY, replay=d)
    assert rel_linf(g["u"], ref) <= TOL["f64"]
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=steps, mode=AT_FREE, record=True, max_ctas=5)
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= L
    ref, _ = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=steps, delay_mode=oracle.REPLAY, replay=rec)
    assert rel_linf(g["u"], ref) <= TOL["f64"]


def test_multiple_calls_and_zero_delay_bound_3d():
    from paper_1911_05769_gb300 import AT_SEEDED, AT_SYNC
    n, sub = 32, (16, 16, 8)
    nu = NU[n]
    u0, dt = case(n, seed=9)
    one = gpu_run3d(u0, sub=sub, L=2, nu=nu, dt=dt, steps=30, mode=AT_SEEDED, seed=2, max_ctas=3)
    two = gpu_run3d(u0, sub=sub, L=2, nu=nu, dt=dt, steps=30, mode=AT_SEEDED, seed=2, max_ctas=3, calls=[11, 19])
    assert np.array_equal(one["u"], two["u"])
    a = gpu_run3d(u0, sub=sub, L=0, nu=nu, dt=dt, steps=20, mode=AT_SEEDED, seed=2)
    b = gpu_run3d(u0, sub=sub, L=0, nu=nu, dt=dt, steps=20, mode=AT_SYNC)
    assert np.array_equal(a["u"], b["u"])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_large_box_3d(dtype):
    """256^3 points in 32^3 subdomains (512 subdomains, the workload's
    subdomain size, k^-5/3 field with |k| <= 32), seeded L = 2, 6 steps,
    against the oracle over the whole box."""
    from paper_1911_05769_gb300 import AT_SEEDED
    n, sub, L, nu = 256, (32, 32, 32), 2, NU[256]
    u0 = W.u0_spectral3d(n, seed=4, kmax=32)
    dt = W.dt_rule(u0, 2 * np.pi / n, nu, dim=3)
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=6, dtype=dtype, mode=AT_SEEDED, seed=5)
    ref, _ = oracle.run3d(u0, P=(8, 8, 8), L=L, nu=nu, dt=dt, n_steps=6, delay_mode=oracle.SEEDED, seed=5)
    assert rel_linf(g["u"], ref) <= TOL[dtype]


def test_workload_parameters_all_2000_steps_3d():
    """The 3D workload's own parameters -- dx = 2 pi / 512, nu = 5e-3, dt by
    the CFL rule (1.0e-3), subdomains of 32^3, L = 2, seeded delays -- over all
    of its 2000 steps, on a periodic 128^3 box of length pi / 2 whose k^-5/3
    field keeps the workload's wavenumbers (|k| <= 32 of the 2 pi box: |k| <= 8
    of this one).  FP32 state within 1e-5 and FP64 within 1e-12 of the FP64
    oracle over the whole box.  (A window of the 512^3 run cannot be checked
    alone: after 2000 steps every point depends on the whole box.)"""
    from paper_1911_05769_gb300 import AT_SEEDED
    n, sub, L, nu, steps = 128, (32, 32, 32), 2, 5e-3, 2000
    box = np.pi / 2
    u0 = W.u0_spectral3d(n, seed=4, kmax=8)
    dx = box / n
    assert abs(dx - 2 * np.pi / 512) < 1e-15
    dt = W.dt_rule(u0, dx, nu, dim=3)
    ref, hist = oracle.run3d(u0, P=(4, 4, 4), L=L, nu=nu, dt=dt, n_steps=steps, length=box,
                             delay_mode=oracle.SEEDED, seed=5)
    assert np.max(np.abs(ref)) > 0.05          # the field is still there after 2000 steps
    for dtype in ("f32", "f64"):
        g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=steps, dtype=dtype, mode=AT_SEEDED, seed=5,
                      length=(box,) * 3)
        assert rel_linf(g["u"], ref) <= TOL[dtype], (dtype, rel_linf(g["u"], ref))
        assert np.array_equal(g["hist"], hist)


def check_pass_structure(rec, passes):
    """Delays of blocked passes: a pass (lv, b) from level lv > 0 of b levels
    gives level lv + j the delay k0 + j on every face (the halo of the pass is
    extrapolated from one pair of levels); the pass from level 0 has one level
    at delay 0."""
    for lv, b in passes:
        if lv == 0:
            assert b == 1 and np.all(rec[0] == 0)
            continue
        for j in range(1, b):
            assert np.array_equal(rec[lv + j].astype(int) - rec[lv].astype(int), np.full(rec[lv].shape, j))


BLOCKED = [
    # (n, sub, L, steps_per_pass, max_ctas, calls)
    (32, (16, 8, 8), 3, 2, 5, None),          # several subdomains per CTA
    (32, (16, 8, 8), 3, 4, 0, None),          # L + 1 levels per pass, one subdomain per CTA
    (32, (32, 32, 16), 2, 3, 3, None),        # planes of 1024 points (every thread busy)
    (24, (8, 4, 3), 2, 3, 7, None),           # planes of 32 points, 3 planes per subdomain
    (32, (16, 16, 8), 2, 3, 0, [7, 12, 17]),  # several calls: passes restart at each call's first level
    (32, (16, 8, 8), 2, 3, 5, [1, 1, 2, 3, 5]),  # calls shorter than a pass (the start-up pass: one level)
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,sub,L,spp,max_ctas,calls", BLOCKED)
def test_blocked_free_3d_replays_in_oracle(dtype, n, sub, L, spp, max_ctas, calls):
    """Free-running passes of steps_per_pass levels: the recorded delays
    (within L, k0 + j over a pass) replayed by the oracle give the kernel's
    result, and the delay histogram is theirs."""
    from paper_1911_05769_gb300 import AT_FREE
    nu = NU[n]
    u0, dt = case(n, seed=11)
    P = tuple(n // m for m in sub)
    steps = sum(calls) if calls else 36
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=steps, dtype=dtype, mode=AT_FREE, record=True,
                  max_ctas=max_ctas, steps_per_pass=spp, calls=calls)
    assert g["info"].steps_per_pass == spp
    assert g["info"].threads == 256              # the blocked kernel's CTAs
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= L
    # passes restart at each call's first level; the pass from level 0 has one level
    passes, lv = [], 0
    for c in (calls or [steps]):
        end = lv + c
        while lv < end:
            b = 1 if lv == 0 else min(spp, end - lv)
            passes.append((lv, b))
            lv += b
    check_pass_structure(rec, passes)
    ref, hist = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=steps, delay_mode=oracle.REPLAY, replay=rec)
    assert rel_linf(g["u"], ref) <= TOL[dtype], rel_linf(g["u"], ref)
    assert np.array_equal(g["hist"], hist)
    assert np.array_equal(np.bincount(rec.ravel(), minlength=L + 1), hist)


def test_blocked_free_3d_mixed_with_other_modes():
    """Blocked free-running calls between seeded and synchronous calls: each
    call finds the ring levels it reads, whatever the previous call's mode."""
    import torch

    from paper_1911_05769_gb300 import AT_FREE, AT_OK, AT_SEEDED, AT_SYNC, Solver3D, binding
    n, sub, L = 32, (16, 8, 8), 3
    nu = NU[n]
    u0, dt = case(n, seed=12)
    P = tuple(n // m for m in sub)
    s = Solver3D((n, n, n), sub, L, nu, dt, dtype="f64", seed=3, max_ctas=6, steps_per_pass=3)
    s.set_state(torch.from_numpy(np.ascontiguousarray(u0).ravel()).cuda())
    recs = []
    for c, mode in ((10, AT_FREE), (7, AT_SEEDED), (9, AT_FREE), (3, AT_SYNC), (8, AT_FREE)):
        d = torch.full((c, s.P, 6), -1, dtype=torch.int8, device="cuda")
        s.step(c, mode, d)
        rec = d.cpu().numpy()
        if mode == AT_SYNC:
            rec[:] = 0
        recs.append(rec)
    rec = np.concatenate(recs, axis=0)
    assert rec.min() >= 0 and rec.max() <= L
    out = torch.empty(s.N, dtype=s.tdtype, device="cuda")
    assert binding.at_state(s.h, out.data_ptr()) == AT_OK, binding.at_last_error()
    s.close()
    ref, _ = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=rec.shape[0], delay_mode=oracle.REPLAY, replay=rec)
    assert rel_linf(out.double().cpu().numpy().reshape(u0.shape), ref) <= TOL["f64"]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,sub", [(32, (16, 8, 8)), (64, (32, 32, 32))])
def test_blocked_free_3d_unequal_spacing(dtype, n, sub):
    """Blocked free-running passes on a box with unequal spacing (z half as
    long: the stepper's per-axis coefficients rather than its equal-spacing
    form; 32^3 subdomains take the instances with compile-time sizes),
    recorded delays replayed by the oracle."""
    from paper_1911_05769_gb300 import AT_FREE
    L, spp = 2, 3
    nu = NU.get(n, 0.05)
    u0 = W.u0_spectral3d(n, seed=13, kmax=8)
    length = (2 * np.pi, 2 * np.pi, np.pi)
    dx = tuple(a / n for a in length)
    dt = W.dt_rule(u0, min(dx), nu, dim=3)
    P = tuple(n // m for m in sub)
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=30, dtype=dtype, mode=AT_FREE, record=True,
                  max_ctas=5 if P[0] * P[1] * P[2] > 8 else 3, steps_per_pass=spp, length=length)
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= L
    ref, hist = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=30, dx=dx, delay_mode=oracle.REPLAY, replay=rec)
    assert rel_linf(g["u"], ref) <= TOL[dtype], rel_linf(g["u"], ref)
    assert np.array_equal(g["hist"], hist)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,sub", [(32, (32, 32, 8)), (64, (32, 32, 32))])
def test_seeded_3d_unequal_spacing(dtype, n, sub):
    """One level per pass on a box of unequal spacing: the per-axis form of
    the stencil (the cubic boxes above take the equal-spacing form; 32^3
    subdomains the instances with compile-time sizes)."""
    from paper_1911_05769_gb300 import AT_SEEDED
    L = 2
    nu = NU.get(n, 0.05)
    u0 = W.u0_spectral3d(n, seed=14, kmax=8)
    length = (2 * np.pi, np.pi, 2 * np.pi)
    dx = tuple(a / n for a in length)
    dt = W.dt_rule(u0, min(dx), nu, dim=3)
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=30, dtype=dtype, mode=AT_SEEDED, seed=6, length=length)
    ref, hist = oracle.run3d(u0, P=tuple(n // m for m in sub), L=L, nu=nu, dt=dt, n_steps=30, dx=dx,
                             delay_mode=oracle.SEEDED, seed=6)
    assert rel_linf(g["u"], ref) <= TOL[dtype], rel_linf(g["u"], ref)
    assert np.array_equal(g["hist"], hist)


def test_workload_parameters_blocked_free_2000_steps_3d():
    """The 3D workload's parameters (as in the seeded test above: dx = 2 pi /
    512, nu = 5e-3, the CFL dt, 32^3 subdomains, L = 2, a 128^3 box of length
    pi / 2) over all 2000 steps, free-running in passes of L + 1 = 3 levels:
    the oracle replaying the recorded delays matches within 1e-5 (FP32) and
    1e-12 (FP64)."""
    from paper_1911_05769_gb300 import AT_FREE
    n, sub, L, nu, steps = 128, (32, 32, 32), 2, 5e-3, 2000
    box = np.pi / 2
    u0 = W.u0_spectral3d(n, seed=4, kmax=8)
    dt = W.dt_rule(u0, box / n, nu, dim=3)
    for dtype in ("f32", "f64"):
        g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=steps, dtype=dtype, mode=AT_FREE, record=True,
                      length=(box,) * 3, steps_per_pass=L + 1)
        rec = g["rec"]
        assert rec.min() >= 0 and rec.max() <= L
        ref, hist = oracle.run3d(u0, P=(4, 4, 4), L=L, nu=nu, dt=dt, n_steps=steps, length=box,
                                 delay_mode=oracle.REPLAY, replay=rec)
        assert np.max(np.abs(ref)) > 0.05
        assert rel_linf(g["u"], ref) <= TOL[dtype], (dtype, rel_linf(g["u"], ref))
        assert np.array_equal(g["hist"], hist)


def _smooth_box(shape, seed):
    """A seeded smooth periodic field on a box of shape (n2, n1, n0): a few
    low Fourier modes with random phases, max |u| = 1 (inputs only)."""
    rng = np.random.default_rng(seed)
    n2, n1, n0 = shape
    z, y, x = np.meshgrid(np.arange(n2) / n2, np.arange(n1) / n1, np.arange(n0) / n0, indexing="ij")
    u = np.zeros(shape)
    for _ in range(6):
        k = rng.integers(0, 3, size=3)
        u += rng.uniform(0.5, 1.0) * np.sin(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + rng.uniform(0, 2 * np.pi))
    return u / np.max(np.abs(u))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape,sub", [((16, 32, 128), (128, 8, 4)),    # rows of 128 points: a row is a warp
                                       ((6, 8, 8), (4, 4, 3))])          # the smallest subdomain
def test_blocked_free_3d_edge_shapes(dtype, shape, sub):
    """Blocked free-running passes on the extreme subdomain shapes the blocked
    stepper takes (sub[0] = 128 and 4), against the oracle replaying the
    recorded delays."""
    from paper_1911_05769_gb300 import AT_FREE
    L, spp = 2, 3
    u0 = _smooth_box(shape, seed=15)
    n2, n1, n0 = shape
    dx = tuple(2 * np.pi / n for n in (n0, n1, n2))
    nu = max(dx) / 2                  # a cell Peclet number of about 2 on the coarsest axis (max |u0| = 1)
    dt = W.dt_rule(u0.ravel(), min(dx), nu, dim=3)
    P = (n0 // sub[0], n1 // sub[1], n2 // sub[2])
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=24, dtype=dtype, mode=AT_FREE, record=True,
                  max_ctas=3, steps_per_pass=spp)
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= L
    ref, hist = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=24, dx=dx, delay_mode=oracle.REPLAY, replay=rec)
    assert np.all(np.isfinite(ref)) and np.max(np.abs(ref)) > 0.01
    assert rel_linf(g["u"], ref) <= TOL[dtype], rel_linf(g["u"], ref)
    assert np.array_equal(g["hist"], hist)


def test_blocked_free_3d_four_levels_on_32_cubes():
    """Passes of 4 levels (L = 3) on 32^3 subdomains: FP32 fits one CTA per
    SM and replays in the oracle; FP64 (24 halo planes of 8 KiB) does not fit
    a CTA's shared memory and at_create refuses it with AT_ERR_RESIDENCY."""
    import paper_1911_05769_gb300 as at
    n, sub, L = 64, (32, 32, 32), 3
    nu = 0.05
    u0 = W.u0_spectral3d(n, seed=16, kmax=8)
    dt = W.dt_rule(u0, 2 * np.pi / n, nu, dim=3)
    g = gpu_run3d(u0, sub=sub, L=L, nu=nu, dt=dt, steps=21, dtype="f32", mode=at.AT_FREE, record=True,
                  steps_per_pass=L + 1)
    ref, _ = oracle.run3d(u0, P=(2, 2, 2), L=L, nu=nu, dt=dt, n_steps=21, delay_mode=oracle.REPLAY, replay=g["rec"])
    assert rel_linf(g["u"], ref) <= TOL["f32"]
    with pytest.raises(at.AtError) as e:
        at.Solver3D((n, n, n), sub, L, nu, dt, dtype="f64", steps_per_pass=L + 1)
    assert e.value.code == at.AT_ERR_RESIDENCY and "shared memory" in str(e.value)
