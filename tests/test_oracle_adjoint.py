"""Pins of the oracle's discrete adjoint (reverse-mode differentiation of the
AT run) against quantities that do not use it: central finite differences of
the forward oracle, and the full Jacobian built column by column from forward
runs on a tiny grid.  A terminal loss J = ||u(T) - u_target||^2 as in the
adjoint workload (its gradient with respect to u(T) is 2 (u(T) - u_target))."""
import numpy as np
import pytest

import at_workloads as W
import oracle


def setup(N=96, P=6, order=2, L=2, nu=0.05, steps=40, seed=3, mode=oracle.SEEDED):
    x, dx = W.grid(N)
    u0 = np.sin(x) + 0.5 * np.sin(3 * x + 1)
    dt = W.dt_rule(u0, dx, nu)
    kw = dict(P=P, order=order, L=L, nu=nu, dt=dt, n_steps=steps, delay_mode=mode, seed=seed)
    if mode == oracle.REPLAY:
        kw["replay"] = W.random_delays(steps, P, L, seed=4)
    rng = np.random.default_rng(seed)
    target = oracle.run(u0 + 0.05 * rng.standard_normal(N), **kw)[0]
    return u0, target, kw


def loss(u0, target, kw, nu=None):
    k2 = dict(kw)
    if nu is not None:
        k2["nu"] = nu
    uT = oracle.run(u0, **k2)[0]
    return float(np.sum((uT - target) ** 2))


@pytest.mark.parametrize("order,L,mode", [(2, 2, oracle.SEEDED), (4, 3, oracle.SEEDED), (2, 0, oracle.SYNC),
                                          (4, 2, oracle.SYNC)])
def test_adjoint_forward_equals_run(order, L, mode):
    u0, target, kw = setup(order=order, L=L, mode=mode)
    ref = oracle.run(u0, **kw)[0]
    uT, _, _ = oracle.adjoint(u0, np.zeros_like(u0), **kw)
    assert np.array_equal(uT, ref)


@pytest.mark.parametrize("order,L,mode", [(2, 2, oracle.SEEDED), (4, 3, oracle.SEEDED), (2, 2, oracle.SYNC)])
def test_adjoint_matches_central_differences(order, L, mode):
    """<dJ/du0, d> against (J(u0 + e d) - J(u0 - e d)) / 2e on random
    directions, and dJ/dnu against the same difference in nu."""
    u0, target, kw = setup(order=order, L=L, mode=mode)
    uT = oracle.run(u0, **kw)[0]
    _, lam0, dnu = oracle.adjoint(u0, 2.0 * (uT - target), **kw)
    rng = np.random.default_rng(11)
    for _ in range(4):
        d = rng.standard_normal(u0.size)
        eps = 1e-5
        fd = (loss(u0 + eps * d, target, kw) - loss(u0 - eps * d, target, kw)) / (2 * eps)
        assert abs(fd - lam0 @ d) <= 1e-7 * max(abs(fd), 1e-12) + 1e-10, (fd, lam0 @ d)
    enu = 1e-6 * kw["nu"]
    fdnu = (loss(u0, target, kw, kw["nu"] + enu) - loss(u0, target, kw, kw["nu"] - enu)) / (2 * enu)
    assert abs(fdnu - dnu) <= 1e-6 * abs(fdnu) + 1e-10, (fdnu, dnu)


def test_adjoint_equals_brute_force_jacobian_transpose():
    """Tiny grid: the Jacobian of u(T) with respect to u0 column by column from
    forward runs (the map is smooth; central differences are exact to
    rounding times the third derivative), then J^T lam against the adjoint."""
    N, P = 16, 4
    u0, target, kw = setup(N=N, P=P, order=2, L=2, steps=6, nu=0.2)
    eps = 1e-6
    Jac = np.empty((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = eps
        Jac[:, c] = (oracle.run(u0 + e, **kw)[0] - oracle.run(u0 - e, **kw)[0]) / (2 * eps)
    lam = np.random.default_rng(2).standard_normal(N)
    _, lam0, _ = oracle.adjoint(u0, lam, **kw)
    assert np.max(np.abs(Jac.T @ lam - lam0)) <= 1e-8 * np.max(np.abs(lam0))


def test_adjoint_of_a_replayed_run_and_standard_weights():
    """Replayed delays, and the negative-control weights (w = (1, 0)) of Fig. 2:
    the adjoint follows whatever forward scheme ran."""
    u0, target, kw = setup(order=2, L=2, mode=oracle.REPLAY)
    for at_w in (True, False):
        k2 = dict(kw, at_weights=at_w)
        uT = oracle.run(u0, **k2)[0]
        _, lam0, _ = oracle.adjoint(u0, 2.0 * (uT - target), **k2)
        d = np.random.default_rng(6).standard_normal(u0.size)
        eps = 1e-5
        fd = (np.sum((oracle.run(u0 + eps * d, **k2)[0] - target) ** 2)
              - np.sum((oracle.run(u0 - eps * d, **k2)[0] - target) ** 2)) / (2 * eps)
        assert abs(fd - lam0 @ d) <= 1e-7 * abs(fd)


def test_adjoint_rejects_what_it_does_not_cover():
    """Only Burgers' equation on the whole periodic domain is differentiated."""
    import ctypes
    u0 = np.zeros(32)
    out = np.empty(32)
    for eq, bc in ((oracle.EQ_LINEAR, oracle.BC_PERIODIC), (oracle.EQ_BURGERS, oracle.BC_TANH)):
        c = oracle.Cfg(N=32, P=4, p_lo=0, p_count=4, order=2, L=1, nu=0.1, dt=1e-3, x0=0.0, dx=0.1,
                       forcing_amp=0.0, eq=eq, bc=bc, adv_c=1.0, tanh_a=0.0, tanh_c=0.0, tanh_xc=0.0,
                       delay_mode=0, per_subdomain=0, at_weights=1, pad_=0, seed=0)
        ptr = u0.ctypes.data_as(ctypes.c_void_p)
        rc = oracle.lib().at_oracle_adjoint(ctypes.byref(c), 2, None, ptr, ptr, None,
                                            out.ctypes.data_as(ctypes.c_void_p), None)
        assert rc != 0
