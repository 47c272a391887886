"""The 3D system of Eq. BS (velocity u, v, w and passive scalars; six-face AT
halos) on the GPU against the system oracle, element by element, and the
device moments against numpy."""
import numpy as np
import pytest

import at_workloads as W
import oracle
from gpu_util import TOL, rel_linf

pytestmark = pytest.mark.gpu


def fields(n, nf, seed=4):
    q = [0.5 * W.u0_spectral3d(n, seed=seed + f, kmax=8) for f in range(nf)]
    return np.stack(q)


def gpu_system(q0, *, sub, L, kappa, dt, steps, dtype="f64", mode=None, seed=0, max_ctas=0, delays=None,
               record=False):
    import torch

    from paper_1911_05769_gb300 import AT_OK, AT_REPLAY, AT_SEEDED, System3D, binding
    mode = AT_SEEDED if mode is None else mode
    nf, n2, n1, n0 = q0.shape
    s = System3D((n0, n1, n2), sub, L, kappa, dt, dtype=dtype, seed=seed, max_ctas=max_ctas)
    s.set_state(torch.from_numpy(np.ascontiguousarray(q0).ravel()).cuda())
    d = None
    if mode == AT_REPLAY:
        d = torch.from_numpy(np.ascontiguousarray(delays)).cuda()
    elif record:
        d = torch.full((steps, s.P, 6), -1, dtype=torch.int8, device="cuda")
    s.step(steps, mode, d)
    out = torch.empty(s.N, dtype=s.tdtype, device="cuda")
    rc = binding.at_state(s.h, out.data_ptr())
    assert rc == AT_OK, binding.at_last_error()
    hist, _, _ = s.delay_stats()
    res = dict(q=out.double().cpu().numpy().reshape(q0.shape), hist=np.array(hist), moments=s.moments(), P=s.P,
               info=s.info())
    if record:
        res["rec"] = d.cpu().numpy()
    s.close()
    return res


def setup(n, nf, nu=0.1, alphas=(0.05, 0.2)):
    q0 = fields(n, nf)
    kappa = [nu, nu, nu] + list(alphas[:nf - 3])
    dx = 2 * np.pi / n
    dt = W.dt_rule(q0[:3].reshape(-1), dx, max(kappa), dim=3)
    return q0, kappa, dt


CASES = [
    # (n, sub, nf, max_ctas)
    (32, (16, 16, 8), 4, 0),
    (32, (16, 16, 8), 5, 3),
    (32, (32, 16, 8), 3, 0),         # two columns per thread
    (24, (8, 4, 3), 4, 5),           # most threads idle, uneven split
]
# FP32 planes of 1024 points: each thread takes a group of 4 consecutive columns
WIDE = [(64, (32, 32, 8), 5, 7), (64, (32, 32, 4), 3, 0)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,sub,nf,max_ctas", CASES)
def test_seeded_system_matches_oracle(dtype, n, sub, nf, max_ctas):
    from paper_1911_05769_gb300 import AT_SEEDED
    q0, kappa, dt = setup(n, nf)
    P = tuple(n // m for m in sub)
    g = gpu_system(q0, sub=sub, L=2, kappa=kappa, dt=dt, steps=30, dtype=dtype, mode=AT_SEEDED, seed=5,
                   max_ctas=max_ctas)
    ref, hist = oracle.run3d_system(q0, kappa=kappa, P=P, L=2, dt=dt, n_steps=30, delay_mode=oracle.SEEDED, seed=5)
    for f in range(nf):
        assert rel_linf(g["q"][f], ref[f]) <= TOL[dtype], f
    assert np.array_equal(g["hist"], hist)
    # device moments of the state against numpy
    for f, (m1, m2) in enumerate(g["moments"]):
        assert abs(m1 - g["q"][f].mean()) <= 1e-12 * max(abs(g["q"][f]).max(), 1e-300)
        assert abs(m2 - (g["q"][f] ** 2).mean()) <= 1e-12 * (g["q"][f] ** 2).mean()


@pytest.mark.parametrize("n,sub,nf,max_ctas", WIDE)
def test_wide_planes_fp32_system(n, sub, nf, max_ctas):
    from paper_1911_05769_gb300 import AT_SEEDED
    q0, kappa, dt = setup(n, nf)
    P = tuple(n // m for m in sub)
    g = gpu_system(q0, sub=sub, L=2, kappa=kappa, dt=dt, steps=30, dtype="f32", mode=AT_SEEDED, seed=5,
                   max_ctas=max_ctas)
    ref, hist = oracle.run3d_system(q0, kappa=kappa, P=P, L=2, dt=dt, n_steps=30, delay_mode=oracle.SEEDED, seed=5)
    for f in range(nf):
        assert rel_linf(g["q"][f], ref[f]) <= TOL["f32"], f
    assert np.array_equal(g["hist"], hist)


def test_sync_replay_and_free_system():
    from paper_1911_05769_gb300 import AT_FREE, AT_REPLAY, AT_SYNC
    n, sub, nf, L = 32, (16, 8, 8), 4, 3
    q0, kappa, dt = setup(n, nf)
    P = tuple(n // m for m in sub)
    NP = P[0] * P[1] * P[2]
    steps = 24
    g = gpu_system(q0, sub=sub, L=L, kappa=kappa, dt=dt, steps=steps, mode=AT_SYNC, max_ctas=4)
    ref, _ = oracle.run3d_system(q0, kappa=kappa, P=P, L=L, dt=dt, n_steps=steps, delay_mode=oracle.SYNC)
    assert rel_linf(g["q"], ref) <= TOL["f64"]
    d = np.random.default_rng(3).integers(0, L + 1, size=(steps, NP, 6), dtype=np.int8)
    g = gpu_system(q0, sub=sub, L=L, kappa=kappa, dt=dt, steps=steps, mode=AT_REPLAY, delays=d)
    ref, _ = oracle.run3d_system(q0, kappa=kappa, P=P, L=L, dt=dt, n_steps=steps, delay_mode=oracle.REPLAY, replay=d)
    assert rel_linf(g["q"], ref) <= TOL["f64"]
    g = gpu_system(q0, sub=sub, L=L, kappa=kappa, dt=dt, steps=steps, mode=AT_FREE, record=True, max_ctas=5)
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= L
    ref, _ = oracle.run3d_system(q0, kappa=kappa, P=P, L=L, dt=dt, n_steps=steps, delay_mode=oracle.REPLAY,
                                 replay=rec)
    assert rel_linf(g["q"], ref) <= TOL["f64"]


def test_equal_velocity_components_match_the_scalar_solver():
    """u = v = w = f: each velocity component of the system follows the scalar
    3D equation, so it matches the scalar solver to rounding."""
    import torch

    from paper_1911_05769_gb300 import AT_SEEDED, Solver3D
    n, sub = 32, (16, 16, 8)
    f = 0.5 * W.u0_spectral3d(n, seed=9, kmax=8)
    nu = 0.1
    dt = W.dt_rule(f.reshape(-1), 2 * np.pi / n, nu, dim=3)
    s = Solver3D((n, n, n), sub, 2, nu, dt, dtype="f64", seed=4)
    s.set_state(torch.from_numpy(f.ravel()).cuda())
    s.step(25, AT_SEEDED)
    ref = s.state().cpu().numpy().reshape(f.shape)
    s.close()
    g = gpu_system(np.stack([f, f, f]), sub=sub, L=2, kappa=[nu, nu, nu], dt=dt, steps=25, mode=AT_SEEDED, seed=4)
    for c in range(3):
        assert rel_linf(g["q"][c], ref) <= TOL["f64"]
