"""Pins of the 3D oracle (scalar Burgers u_t + u (u_x + u_y + u_z) = nu lap u,
and the system of Eq. BS with velocity (u, v, w) and passive scalars; order 2,
AT halos on the six faces of every subdomain) against things that do not use
it: the 1D oracle, plain Python restatements on tiny boxes, the scalar
equation (system with u = v = w), the exact Cole-Hopf solution along the
diagonal, and the exact decaying mode of a scalar in a uniform flow."""
import math

import numpy as np
import pytest

import at_workloads as W
import oracle


def test_field_constant_in_y_and_z_equals_the_1d_run():
    """With u0 = u0(x) and zero delays on the y and z faces, every y and z
    difference is exactly zero, so the 3D run equals the 1D run with the same
    x-face delays bit for bit."""
    n0, n1, n2, P0 = 64, 8, 4, 8
    steps = 30
    x, dx = W.grid(n0)
    f = np.sin(x) + 0.5 * np.sin(3 * x + 1)
    nu = 0.05
    dt = W.dt_rule(f, dx, nu, dim=3)
    d1 = W.random_delays(steps, P0, 2, seed=5)
    ref, _ = oracle.run(f, P=P0, order=2, L=2, nu=nu, dt=dt, n_steps=steps, delay_mode=oracle.REPLAY, replay=d1)
    P = (P0, 2, 2)
    NP = P0 * 4
    d3 = np.zeros((steps, NP, 6), dtype=np.int8)
    for p in range(NP):
        d3[:, p, 0:2] = d1[:, p % P0, :]
    u0 = np.broadcast_to(f, (n2, n1, n0)).copy()
    out, _ = oracle.run3d(u0, P=P, L=2, nu=nu, dt=dt, n_steps=steps, dx=(dx, 0.3, 0.7), delay_mode=oracle.REPLAY,
                          replay=d3)
    for k in range(n2):
        for j in range(n1):
            assert np.array_equal(out[k, j], ref)


def brute_force_3d(u0, P, L, nu, dt, steps, dx, seed):
    """Plain restatement: per level, per point, per axis, the two neighbours,
    each either a value at level n or (across a face) (k+1) f^{n-k} - k f^{n-k-1}."""
    n2, n1, n0 = u0.shape
    n = (n0, n1, n2)
    m = tuple(n[a] // P[a] for a in range(3))
    NP = P[0] * P[1] * P[2]
    hist = [u0.copy()]
    for lev in range(steps):
        cur = hist[-1]
        new = np.empty_like(cur)
        for k in range(n2):
            for j in range(n1):
                for i in range(n0):
                    c = (i, j, k)
                    p = ((k // m[2]) * P[1] + j // m[1]) * P[0] + i // m[0]
                    u = cur[k, j, i]
                    d1 = d2 = 0.0
                    for a in range(3):
                        vals = []
                        for side, off in ((0, -1), (1, 1)):
                            q = list(c)
                            q[a] = (c[a] + off) % n[a]
                            loc = c[a] % m[a] + off
                            if 0 <= loc < m[a]:
                                vals.append(cur[q[2], q[1], q[0]])
                                continue
                            face = 2 * a + side
                            kr = oracle.seeded_delay(seed, lev, p, NP, face, 6, L)
                            kf = min(kr, max(0, lev - 1))
                            if kf == 0:
                                vals.append(hist[lev][q[2], q[1], q[0]])
                            else:
                                vals.append((kf + 1) * hist[lev - kf][q[2], q[1], q[0]]
                                            - kf * hist[lev - kf - 1][q[2], q[1], q[0]])
                        d1 += (vals[1] - vals[0]) / (2 * dx[a])
                        d2 += (vals[1] - 2 * u + vals[0]) / dx[a] ** 2
                    new[k, j, i] = u + dt * (-u * d1 + nu * d2)
        hist.append(new)
    return hist[-1]


def test_brute_force_on_a_tiny_box():
    rng = np.random.default_rng(8)
    u0 = rng.standard_normal((4, 6, 4))
    P, L, nu, dt, steps, dx = (2, 3, 2), 2, 0.3, 1e-3, 6, (0.5, 0.4, 0.6)
    ref = brute_force_3d(u0, P, L, nu, dt, steps, dx, seed=4)
    out, _ = oracle.run3d(u0, P=P, L=L, nu=nu, dt=dt, n_steps=steps, dx=dx, delay_mode=oracle.SEEDED, seed=4)
    assert np.max(np.abs(out - ref)) <= 1e-14 * np.max(np.abs(ref))


def cole_hopf_diagonal(n, t, nu, a=2.0):
    """u = G(x + y + z, t) / 3 with G the Cole-Hopf solution of
    G_t + G G_xi = 3 nu G_xixi: G = 2 nu' e^{-nu' t} sin xi / (a + e^{-nu' t} cos xi), nu' = 3 nu."""
    x, _ = W.grid(n)
    xi = x[None, None, :] + x[None, :, None] + x[:, None, None]
    nup = 3.0 * nu
    e = math.exp(-nup * t)
    return 2.0 * nup * e * np.sin(xi) / (a + e * np.cos(xi)) / 3.0


@pytest.mark.parametrize("mode", [oracle.SYNC, oracle.SEEDED])
def test_convergence_to_cole_hopf_along_the_diagonal(mode):
    """Second order in space with dt ~ dx^2 (forward Euler's O(dt) is O(dx^2)),
    with and without delays (Eq. AT1/AT2 keep the AT scheme at second order)."""
    nu, T = 0.1, 0.25
    errs = []
    for n in (16, 32):
        dx = 2 * math.pi / n
        steps = int(round(T / (0.05 * dx * dx / nu)))
        dt = T / steps
        u0 = cole_hopf_diagonal(n, 0.0, nu)
        out, _ = oracle.run3d(u0, P=(4, 4, 4), L=2, nu=nu, dt=dt, n_steps=steps, delay_mode=mode, seed=3)
        errs.append(float(np.max(np.abs(out - cole_hopf_diagonal(n, T, nu)))))
    assert 3.3 < errs[0] / errs[1] < 4.8, errs


def test_zero_delay_bound_equals_synchronous_and_histogram():
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal((8, 8, 8))
    kw = dict(P=(2, 2, 2), nu=0.2, dt=1e-3, n_steps=10)
    a, ha = oracle.run3d(u0, L=0, delay_mode=oracle.SEEDED, seed=9, **kw)
    b, _ = oracle.run3d(u0, L=0, delay_mode=oracle.SYNC, **kw)
    assert np.array_equal(a, b)
    assert ha.tolist() == [10 * 8 * 6]
    _, h2 = oracle.run3d(u0, L=2, delay_mode=oracle.SEEDED, seed=9, **kw)
    assert h2.sum() == 10 * 8 * 6 and h2[1] > 0 and h2[2] > 0


# ---- the system of Eq. BS: velocity (u, v, w) and passive scalars ----------

def test_system_with_equal_velocity_components_is_the_scalar_equation():
    """u = v = w = f makes every velocity component obey
    f_t + f (f_x + f_y + f_z) = nu lap f, the scalar 3D equation."""
    rng = np.random.default_rng(2)
    f = 0.3 * rng.standard_normal((8, 8, 8))
    kw = dict(P=(2, 2, 2), L=2, dt=2e-3, n_steps=12, delay_mode=oracle.SEEDED, seed=6)
    nu = 0.2
    ref, h1 = oracle.run3d(f, nu=nu, **kw)
    q0 = np.stack([f, f, f, f])
    out, h2 = oracle.run3d_system(q0, kappa=[nu, nu, nu, nu], **kw)
    for c in range(4):
        assert np.max(np.abs(out[c] - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.array_equal(h1, h2)


@pytest.mark.parametrize("mode", [oracle.SYNC, oracle.SEEDED])
def test_passive_scalar_in_a_uniform_flow_converges(mode):
    """Constant velocity (c0, c1, c2) stays exactly constant; a scalar
    phi = sin(x + 2y - z) then obeys linear advection-diffusion, exact solution
    exp(-6 alpha t) sin(x + 2y - z - (c0 + 2 c1 - c2) t).  Second order with
    dt ~ dx^2, with and without delays (Eq. AT1/AT2)."""
    c0, c1, c2, alpha, T = 0.3, -0.2, 0.1, 0.05, 0.2
    errs = []
    for n in (16, 32):
        x, dx = W.grid(n)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        phase = X + 2 * Y - Z
        steps = int(round(T / (0.05 * dx * dx / alpha)))
        dt = T / steps
        q0 = np.stack([np.full_like(X, c0), np.full_like(X, c1), np.full_like(X, c2), np.sin(phase)])
        out, _ = oracle.run3d_system(q0, kappa=[0.01, 0.01, 0.01, alpha], P=(4, 4, 4), L=2, dt=dt, n_steps=steps,
                                     delay_mode=mode, seed=3)
        for a in range(3):   # constant velocity stays constant (to rounding of (k+1) c - k c)
            assert np.max(np.abs(out[a] - q0[a])) <= 1e-13
        exact = np.exp(-6 * alpha * T) * np.sin(phase - (c0 + 2 * c1 - c2) * T)
        errs.append(float(np.max(np.abs(out[3] - exact))))
    assert 3.3 < errs[0] / errs[1] < 4.8, errs


def test_system_brute_force_on_a_tiny_box():
    rng = np.random.default_rng(12)
    nf = 5
    q0 = 0.5 * rng.standard_normal((nf, 4, 6, 4))
    kappa = [0.2, 0.2, 0.2, 0.05, 0.4]
    P, L, dt, steps, dx = (2, 3, 2), 2, 1e-3, 5, (0.5, 0.4, 0.6)
    seed = 8
    n2, n1, n0 = q0.shape[1:]
    n = (n0, n1, n2)
    m = tuple(n[a] // P[a] for a in range(3))
    NP = P[0] * P[1] * P[2]
    hist = [q0.copy()]
    for lev in range(steps):
        cur = hist[-1]
        new = np.empty_like(cur)
        for k in range(n2):
            for j in range(n1):
                for i in range(n0):
                    c = (i, j, k)
                    p = ((k // m[2]) * P[1] + j // m[1]) * P[0] + i // m[0]
                    vel = [cur[a, k, j, i] for a in range(3)]
                    for fld in range(nf):
                        q = cur[fld, k, j, i]
                        adv = lap = 0.0
                        for a in range(3):
                            vals = []
                            for side, off in ((0, -1), (1, 1)):
                                qq = list(c)
                                qq[a] = (c[a] + off) % n[a]
                                loc = c[a] % m[a] + off
                                if 0 <= loc < m[a]:
                                    vals.append(cur[fld, qq[2], qq[1], qq[0]])
                                    continue
                                kr = oracle.seeded_delay(seed, lev, p, NP, 2 * a + side, 6, L)
                                kf = min(kr, max(0, lev - 1))
                                h0 = hist[lev - kf][fld, qq[2], qq[1], qq[0]]
                                vals.append(h0 if kf == 0 else (kf + 1) * h0 - kf * hist[lev - kf - 1][fld, qq[2], qq[1], qq[0]])
                            adv += vel[a] * (vals[1] - vals[0]) / (2 * dx[a])
                            lap += (vals[1] - 2 * q + vals[0]) / dx[a] ** 2
                        new[fld, k, j, i] = q + dt * (-adv + kappa[fld] * lap)
        hist.append(new)
    out, _ = oracle.run3d_system(q0, kappa=kappa, P=P, L=L, dt=dt, n_steps=steps, dx=dx, delay_mode=oracle.SEEDED,
                                 seed=seed)
    assert np.max(np.abs(out - hist[-1])) <= 1e-14 * np.max(np.abs(hist[-1]))
