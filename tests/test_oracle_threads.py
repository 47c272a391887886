"""The oracle's thread count changes no result: its point loops share out
whole subdomains (1D) or planes (3D), and every point is computed by the
same arithmetic whatever thread computes it.  Results with one thread and
with every host core must be equal bit for bit."""
import os

import numpy as np

import at_workloads as W
import oracle


def _both(fn):
    before = oracle.threads()
    try:
        oracle.threads(1)
        one = fn()
        oracle.threads(max(2, os.cpu_count() or 2))
        many = fn()
    finally:
        oracle.threads(before)
    return one, many


def test_1d_runs_do_not_depend_on_the_thread_count():
    N, P = 4096, 64
    x, dx = W.grid(N)
    u0 = W.u0_fourier(N, modes=16, seed=2)
    nu = 1e-2
    dt = W.dt_rule(u0, dx, nu)

    def runs():
        a, ha, ka = oracle.run(u0, P=P, order=4, L=3, nu=nu, dt=dt, n_steps=60, forcing_amp=0.1,
                               delay_mode=oracle.SEEDED, seed=3, want_k=True)
        win = u0[5 * (N // P): 25 * (N // P)]
        b, hb = oracle.run(win, N=N, P=P, p_lo=5, p_count=20, order=2, L=2, nu=nu, dt=dt, n_steps=40,
                           delay_mode=oracle.SEEDED, seed=9)
        return a, ha, ka, b, hb

    one, many = _both(runs)
    for x1, x2 in zip(one, many):
        assert np.array_equal(x1, x2)


def test_ensemble_instance_run_does_not_depend_on_the_thread_count():
    inst = W.ensemble(n_inst=3, seed=6)[1]
    u0 = W.instance_field(inst)
    P = inst["n"] // 256

    def runs():
        return oracle.run(u0, P=P, order=2, L=inst["L"], nu=inst["nu"], dt=inst["dt"], n_steps=50,
                          x0=inst["origin"], length=inst["length"], bc=oracle.BC_TANH,
                          tanh=(inst["tanh_a"], inst["tanh_c"], inst["tanh_xc"]),
                          delay_mode=oracle.SEEDED, seed=inst["seed"])

    one, many = _both(runs)
    assert np.array_equal(one[0], many[0]) and np.array_equal(one[1], many[1])


def test_3d_runs_do_not_depend_on_the_thread_count():
    n = 16
    u0 = W.u0_spectral3d(n, seed=4, kmax=4)
    q0 = np.stack([u0, 0.5 * np.roll(u0, 3, axis=0), np.roll(u0, 5, axis=2), u0 ** 2])
    dx = 2 * np.pi / n
    nu = 0.05
    dt = W.dt_rule(u0, dx, nu, dim=3)

    def runs():
        a, ha = oracle.run3d(u0, P=(2, 2, 4), L=2, nu=nu, dt=dt, n_steps=12, delay_mode=oracle.SEEDED, seed=5)
        b, hb = oracle.run3d_system(q0, kappa=[nu, nu, nu, 0.02], P=(4, 2, 2), L=2, dt=dt, n_steps=8,
                                    delay_mode=oracle.SEEDED, seed=6)
        return a, ha, b, hb

    one, many = _both(runs)
    for x1, x2 in zip(one, many):
        assert np.array_equal(x1, x2)
