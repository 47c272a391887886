"""Pins of the CPU oracle against what the paper and the mathematics fix.

No test here retypes the oracle's own formula: each compares it with a
published value, a closed-form solution, an exact identity, an independent
brute-force restatement of Eq. AT1 / AT2, or a convergence rate the paper
states.  Together they are chosen so that a dropped term, a wrong sign, a
wrong index, a wrong time level or a transposed operand fails at least one.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import at_workloads as W
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Delay generator
# --------------------------------------------------------------------------
def test_splitmix64_published_outputs():
    for idx, hexval in _read_table("splitmix64_seed0.txt"):
        assert oracle.splitmix64(0, int(idx)) == int(hexval, 16)


def test_seeded_delay_range_and_uniformity():
    for L in (0, 1, 2, 3, 10):
        ks = np.array([oracle.seeded_delay(7, n, p, 64, f, 2, L)
                       for n in range(40) for p in range(64) for f in range(2)])
        assert ks.min() >= 0 and ks.max() <= L
        if L > 0:
            counts = np.bincount(ks, minlength=L + 1)
            expect = ks.size / (L + 1)
            # every value appears, none deviates by more than 6 sigma
            assert np.all(np.abs(counts - expect) < 6 * math.sqrt(expect))


# --------------------------------------------------------------------------
# AT coefficients (Eq. AT1 / AT2)
# --------------------------------------------------------------------------
def test_weights_match_eq_at1():
    for k, w0, w1 in _read_table("at_weights_eq_at1.txt"):
        w = oracle.weights(2, int(k))
        assert w[0] == float(w0) and w[1] == float(w1)


@pytest.mark.parametrize("s", [2, 3])
def test_weights_reproduce_polynomials_in_time(s):
    """sum_m w_m(k) t_m^q = 0^q for q < s with t_m = -k-m (exact rationals),
    and the identity fails at q = s (the extrapolation is exactly order s)."""
    for k in range(0, 11):
        w = [Fraction(x) for x in oracle.weights(s, k)]
        t = [Fraction(-k - m) for m in range(s)]
        for q in range(s):
            assert sum(wm * tm ** q for wm, tm in zip(w, t)) == (1 if q == 0 else 0)
        if k > 0:
            assert sum(wm * tm ** s for wm, tm in zip(w, t)) != 0


@pytest.mark.parametrize("s", [2, 3])
def test_weights_k0_are_standard(s):
    """Sec. 3.2: for k = 0 the AT schemes reduce to the standard ones."""
    assert list(oracle.weights(s, 0)) == [1.0] + [0.0] * (s - 1)
    lev = np.array([0.3, 17.0, -4.0])[:s]
    assert oracle.extrapolate(s, 0, lev) == 0.3


# --------------------------------------------------------------------------
# Spatial operators: exactness on polynomials and Taylor residual orders
# --------------------------------------------------------------------------
@pytest.mark.parametrize("order,deg1,deg2", [(2, 2, 3), (4, 4, 5)])
def test_central_differences_exact_on_polynomials(order, deg1, deg2):
    """Order-r central first/second differences are exact for polynomials of
    degree <= r (first) and <= r+1 (second, by symmetry)."""
    rng = np.random.default_rng(0)
    R = order // 2
    dx = 0.37
    xc = 0.9
    x = xc + dx * np.arange(-R, R + 1)
    for deg, which in ((deg1, 0), (deg2, 1)):
        c = rng.normal(size=deg + 1)
        p = np.polynomial.Polynomial(c)
        d1, d2 = oracle.derivs(order, p(x), dx)
        exact = p.deriv(1)(xc) if which == 0 else p.deriv(2)(xc)
        got = d1 if which == 0 else d2
        assert abs(got - exact) <= 1e-11 * (1 + abs(exact))
    # one degree more breaks exactness of the first difference (order is sharp)
    p = np.polynomial.Polynomial([0] * (deg1 + 1) + [1.0])
    d1, _ = oracle.derivs(order, p(x), dx)
    assert abs(d1 - p.deriv(1)(xc)) > 1e-6


def _at_point(order, k, side, f, xi, tn, dx, dt):
    """AT derivatives at a subdomain-boundary point x_i, level n, using the
    oracle's halo approximation and stencil; the R points beyond the boundary
    (left if side == 0) are taken from levels n-k-m."""
    R, s = order // 2, order // 2 + 1
    v = []
    for j in range(-R, R + 1):
        xj = xi + j * dx
        remote = (j < 0) if side == 0 else (j > 0)
        if remote:
            lev = [f(xj, tn - (k + m) * dt) for m in range(s)]
            v.append(oracle.extrapolate(s, k, lev))
        else:
            v.append(f(xj, tn))
    return oracle.derivs(order, np.array(v), dx)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("side", [0, 1])
def test_at_operator_exact_on_space_time_polynomials(order, side):
    """f(x,t) polynomial of degree <= order in x and < s in t: the AT
    derivatives (Eq. AT1/AT2 and the order-4 reading) are exact."""
    rng = np.random.default_rng(order * 10 + side)
    s = order // 2 + 1
    C = rng.normal(size=(order + 1, s))

    def f(x, t):
        return sum(C[a, b] * x ** a * t ** b for a in range(order + 1) for b in range(s))

    def fx(x, t):
        return sum(a * C[a, b] * x ** (a - 1) * t ** b for a in range(1, order + 1) for b in range(s))

    def fxx(x, t):
        return sum(a * (a - 1) * C[a, b] * x ** (a - 2) * t ** b for a in range(2, order + 1) for b in range(s))

    for k in range(0, 4):
        d1, d2 = _at_point(order, k, side, f, 0.3, 0.8, 0.21, 0.05)
        assert abs(d1 - fx(0.3, 0.8)) < 1e-9 * (1 + abs(fx(0.3, 0.8)))
        assert abs(d2 - fxx(0.3, 0.8)) < 1e-8 * (1 + abs(fxx(0.3, 0.8)))


@pytest.mark.parametrize("order", [2, 4])
def test_standard_stencil_truncation_order(order):
    """k = 0 (the standard scheme): f = sin(x - t), errors of f_x and f_xx
    decay as dx^order."""
    f = lambda x, t: math.sin(x - t)
    dxs = [0.1 / 2 ** j for j in range(4)]
    e1, e2 = [], []
    for dx in dxs:
        d1, d2 = _at_point(order, 0, 0, f, 0.4, 1.0, dx, dx * dx)
        e1.append(abs(d1 - math.cos(0.4 - 1.0)))
        e2.append(abs(d2 + math.sin(0.4 - 1.0)))
    s1 = np.polyfit(np.log(dxs), np.log(e1), 1)[0]
    s2 = np.polyfit(np.log(dxs), np.log(e2), 1)[0]
    assert abs(s1 - order) < 0.2 and abs(s2 - order) < 0.2, (s1, s2)


@pytest.mark.parametrize("order", [2, 4])
def test_asynchrony_error_terms(order):
    """The part of the AT derivative error due to the delay (AT minus the
    k = 0 result at the same point), with dt = dx^2.  Order 2, Eq. AT1: the
    halo error is k(k+1) dt^2 f_tt / 2, so f_xx gains O(k(k+1) dt^2/dx^2) =
    O(dx^2) and f_x gains O(dt^2/dx) = O(dx^3).  Order 4 (quadratic
    extrapolation): halo error k(k+1)(k+2) dt^3 f_ttt / 6, giving O(dx^4) in
    f_xx and O(dx^5) in f_x.  The k dependence is checked as well."""
    f = lambda x, t: math.sin(x - t)
    dxs = [0.1 / 2 ** j for j in range(4)]
    want1, want2 = (3.0, 2.0) if order == 2 else (5.0, 4.0)
    kfac = (lambda k: k * (k + 1)) if order == 2 else (lambda k: k * (k + 1) * (k + 2))
    amp = {}
    for k in (1, 3):
        a1, a2 = [], []
        for dx in dxs:
            dt = dx * dx
            d1, d2 = _at_point(order, k, 0, f, 0.4, 1.0, dx, dt)
            s1, s2 = _at_point(order, 0, 0, f, 0.4, 1.0, dx, dt)
            a1.append(abs(d1 - s1))
            a2.append(abs(d2 - s2))
        p1 = np.polyfit(np.log(dxs), np.log(a1), 1)[0]
        p2 = np.polyfit(np.log(dxs), np.log(a2), 1)[0]
        assert abs(p1 - want1) < 0.25 and abs(p2 - want2) < 0.25, (k, p1, p2)
        amp[k] = a2[-1]
    ratio = amp[3] / amp[1]
    assert abs(ratio / (kfac(3) / kfac(1)) - 1.0) < 0.05, ratio


# --------------------------------------------------------------------------
# Brute force: Eq. AT1 / AT2 as printed (order 2), dense history
# --------------------------------------------------------------------------
def _brute_force_at1_at2(u0, P, L, nu, dt, dx, delays, n_steps):
    """Independent restatement: f_x, f_xx at the first point of a subdomain by
    Eq. AT1 (delay on the left), at the last point by Eq. AT2 (delay on the
    right), standard central differences elsewhere; delays clamped so that no
    level below 0 is used; forward Euler."""
    N = len(u0)
    M = N // P
    hist = [list(map(float, u0))]
    for n in range(n_steps):
        u = hist[n]
        new = [0.0] * N
        for p in range(P):
            kl = min(int(delays[n, p, 0]), max(0, n - 1))
            kr = min(int(delays[n, p, 1]), max(0, n - 1))
            for m in range(M):
                i = p * M + m
                ip, im = (i + 1) % N, (i - 1) % N
                if m == 0 and M > 1:
                    a, b = hist[n - kl][im], hist[n - kl - 1][im] if kl > 0 else 0.0
                    fx = (u[ip] - (kl + 1) * a + kl * b) / (2 * dx)
                    fxx = (u[ip] - 2 * u[i] + (kl + 1) * a - kl * b) / dx ** 2
                elif m == M - 1:
                    a, b = hist[n - kr][ip], hist[n - kr - 1][ip] if kr > 0 else 0.0
                    fx = ((kr + 1) * a - kr * b - u[im]) / (2 * dx)
                    fxx = ((kr + 1) * a - kr * b - 2 * u[i] + u[im]) / dx ** 2
                else:
                    fx = (u[ip] - u[im]) / (2 * dx)
                    fxx = (u[ip] - 2 * u[i] + u[im]) / dx ** 2
                new[i] = u[i] + dt * (-u[i] * fx + nu * fxx)
        hist.append(new)
    return np.array(hist[-1])


@pytest.mark.parametrize("P,L", [(6, 2), (4, 3), (8, 1)])
def test_oracle_matches_brute_force_eq_at1_at2(P, L):
    N = 48
    x, dx = W.grid(N)
    u0 = np.sin(x) + 0.4 * np.cos(2 * x + 0.3)
    nu = 0.05
    dt = W.dt_rule(u0, dx, nu)
    n_steps = 40
    delays = W.random_delays(n_steps, P, L, seed=P * 100 + L)
    bf = _brute_force_at1_at2(u0, P, L, nu, dt, dx, delays, n_steps)
    u, hist = oracle.run(u0, P=P, order=2, L=L, nu=nu, dt=dt, n_steps=n_steps,
                         delay_mode=oracle.REPLAY, replay=delays)
    assert np.max(np.abs(u - bf)) <= 1e-13 * np.max(np.abs(bf))
    assert hist.sum() == n_steps * P * 2
    # the delays really were exercised
    assert hist[1:].sum() > 0


# --------------------------------------------------------------------------
# Brute force: the order-4 AT scheme (reading c2), dense history
# --------------------------------------------------------------------------
def _brute_force_order4(u0, P, L, nu, dt, dx, delays, n_steps, A=0.0, x0=0.0):
    """Independent restatement of the fourth-order AT run: every halo value
    across a face is the quadratic Lagrange extrapolation in time of the
    neighbour's levels n-k, n-k-1, n-k-2 to level n, weights
    ((k+1)(k+2)/2, -k(k+2), k(k+1)/2); both halo points of a face (offsets
    1 and 2 beyond the subdomain) take that face's delay.  Delays are clamped
    to max(0, n - 2) so that no level below 0 is read (Algorithm 2 start-up).
    Then the five-point central differences for f_x and f_xx, the right-hand
    side -u f_x + nu f_xx + A sin x of Eq. BS (forced), forward Euler."""
    N = len(u0)
    M = N // P
    hist = [list(map(float, u0))]
    for n in range(n_steps):
        u = hist[n]
        new = [0.0] * N
        for p in range(P):
            k_face = [min(int(delays[n, p, f]), max(0, n - 2)) for f in (0, 1)]
            for m in range(M):
                i = p * M + m
                v = {}
                for j in (-2, -1, 0, 1, 2):
                    q = i + j
                    inside = p * M <= q < (p + 1) * M
                    qq = q % N
                    if inside:
                        v[j] = u[qq]
                        continue
                    k = k_face[0] if q < p * M else k_face[1]
                    lev = [hist[n - k - mm][qq] if n - k - mm >= 0 else 0.0 for mm in range(3)]
                    w0 = (k + 1) * (k + 2) / 2.0
                    w1 = -k * (k + 2.0)
                    w2 = k * (k + 1) / 2.0
                    v[j] = w0 * lev[0] + w1 * lev[1] + w2 * lev[2]
                fx = (-v[2] + 8.0 * v[1] - 8.0 * v[-1] + v[-2]) / (12.0 * dx)
                fxx = (-v[2] + 16.0 * v[1] - 30.0 * v[0] + 16.0 * v[-1] - v[-2]) / (12.0 * dx * dx)
                x = x0 + i * dx
                new[i] = u[i] + dt * (-v[0] * fx + nu * fxx + A * math.sin(x))
        hist.append(new)
    return np.array(hist[-1])


@pytest.mark.parametrize("P,L,M,A", [(6, 2, 8, 0.0), (4, 3, 12, 0.1), (8, 1, 4, 0.1), (3, 3, 16, 0.0)])
def test_oracle_order4_matches_brute_force_dense_history(P, L, M, A):
    """The order-4 delayed run as a whole (the scheme of the 2^26-point
    workload): replayed random delays, every face, start-up clamp, forcing;
    M = 4 puts both halo points of a face in the neighbour's first/last two."""
    N = P * M
    x, dx = W.grid(N)
    u0 = np.sin(x) + 0.4 * np.cos(2 * x + 0.3) + 0.1 * np.sin(5 * x + 1.0)
    nu = 0.05
    dt = W.dt_rule(u0, dx, nu)
    n_steps = 30
    delays = W.random_delays(n_steps, P, L, seed=P * 1000 + L * 10 + M)
    bf = _brute_force_order4(u0, P, L, nu, dt, dx, delays, n_steps, A=A)
    u, hist = oracle.run(u0, P=P, order=4, L=L, nu=nu, dt=dt, n_steps=n_steps, forcing_amp=A,
                         delay_mode=oracle.REPLAY, replay=delays)
    assert np.max(np.abs(u - bf)) <= 1e-13 * np.max(np.abs(bf))
    assert hist.sum() == n_steps * P * 2
    # the delays were exercised, up to the bound (k >= 2 weights the third level)
    assert hist[1:].sum() > 0 and hist[L] > 0


def test_k0_is_bitwise_synchronous():
    """Sec. 3.2: with every delay 0 the AT run is the synchronous run,
    bit for bit (replayed zeros, and seeded delays with L = 0)."""
    N, P = 256, 8
    x, dx = W.grid(N)
    u0 = W.u0_two_modes(N)
    nu = 0.02
    dt = W.dt_rule(u0, dx, nu)
    for order in (2, 4):
        us, _ = oracle.run(u0, P=P, order=order, L=2, nu=nu, dt=dt, n_steps=200)
        uz, _ = oracle.run(u0, P=P, order=order, L=2, nu=nu, dt=dt, n_steps=200,
                           delay_mode=oracle.REPLAY, replay=np.zeros((200, P, 2), np.int8))
        u0s, _ = oracle.run(u0, P=P, order=order, L=0, nu=nu, dt=dt, n_steps=200,
                            delay_mode=oracle.SEEDED, seed=11)
        assert np.array_equal(us, uz) and np.array_equal(us, u0s)


def test_start_up_clamp():
    """No level below 0 is read: the delays recorded at level n never exceed
    n - s + 1 (Algorithm 2 synchronises while the buffers fill)."""
    for order in (2, 4):
        s = order // 2 + 1
        _, _, k = oracle.run(W.u0_two_modes(64), P=4, order=order, L=5, nu=0.01, dt=1e-4,
                             n_steps=12, delay_mode=oracle.SEEDED, seed=5, want_k=True)
        for n in range(12):
            assert k[n].max() <= max(0, n - s + 1)
        assert k.max() == 5


# --------------------------------------------------------------------------
# Closed forms of the discrete and the continuous problem
# --------------------------------------------------------------------------
@pytest.mark.parametrize("order", [2, 4])
def test_linear_scheme_matches_discrete_fourier_solution(order):
    """Synchronous scheme on u_t + c u_x = nu u_xx, u0 = sin(kappa x): every
    Fourier mode is an eigenvector of the central stencils, so the discrete
    solution is Im(G^n e^{i kappa x}) with G = 1 + dt (-c l1 + nu l2) and
    l1, l2 the Fourier symbols of the first and second difference."""
    N, kappa, c, nu = 64, 3, 0.7, 0.05
    x, dx = W.grid(N)
    th = kappa * dx
    if order == 2:
        l1 = 1j * math.sin(th) / dx
        l2 = -4.0 * math.sin(th / 2) ** 2 / dx ** 2
    else:
        l1 = 1j * (8 * math.sin(th) - math.sin(2 * th)) / (6 * dx)
        l2 = (-2 * math.cos(2 * th) + 32 * math.cos(th) - 30) / (12 * dx ** 2)
    dt = 0.2 * dx * dx / nu
    n = 300
    G = 1 + dt * (-c * l1 + nu * l2)
    exact = np.imag(G ** n * np.exp(1j * kappa * x))
    u, _ = oracle.run(np.sin(kappa * x), P=4, order=order, L=0, nu=nu, dt=dt, n_steps=n,
                      eq=oracle.EQ_LINEAR, adv_c=c)
    assert np.max(np.abs(u - exact)) < 1e-12


def test_forcing_term():
    """With no advection and no diffusion the field grows by n dt A sin(x)."""
    N, A, dt, n = 128, 0.1, 1e-3, 50
    x, dx = W.grid(N)
    u, _ = oracle.run(np.zeros(N), P=4, order=4, L=0, nu=0.0, dt=dt, n_steps=n, eq=oracle.EQ_LINEAR,
                      adv_c=0.0, forcing_amp=A)
    assert np.max(np.abs(u - n * dt * A * np.sin(x))) < 1e-15


def _cole_hopf(x, t, nu, a):
    """Periodic Burgers solution by the Cole-Hopf transform u = -2 nu phi_x/phi,
    phi = a + e^{-nu t} cos x (a heat-equation solution, a > 1)."""
    e = np.exp(-nu * t)
    return 2.0 * nu * e * np.sin(x) / (a + e * np.cos(x))


def _conv_run(N, order, *, P, L, mode, T, nu, lam, dt_pow=2, at_weights=True, seed=3):
    x, dx = W.grid(N)
    a = 1.5
    u0 = _cole_hopf(x, 0.0, nu, a)
    dt0 = lam * dx ** dt_pow
    n = int(math.ceil(T / dt0))
    dt = T / n
    u, _ = oracle.run(u0, P=P, order=order, L=L, nu=nu, dt=dt, n_steps=n, delay_mode=mode,
                      seed=seed, at_weights=at_weights)
    return np.mean(np.abs(u - _cole_hopf(x, T, nu, a)))


def test_burgers_sync_converges_second_order():
    """Closed-form Cole-Hopf solution: slope -2 under dt ~ dx^2 (Sec. 3.2)."""
    for order in (2, 4):
        e = [_conv_run(N, order, P=4, L=0, mode=oracle.SYNC, T=0.5, nu=0.1, lam=1.0) for N in (64, 128, 256)]
        rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        assert np.all(rates > 1.8) and np.all(rates < 2.3), (order, rates)


def test_burgers_order4_converges_fourth_order_with_dt_dx4():
    """Forward Euler adds O(dt); with dt ~ dx^4 the 4th-order stencil's
    spatial order shows: slope -4."""
    e = [_conv_run(N, 4, P=4, L=0, mode=oracle.SYNC, T=0.05, nu=0.1, lam=2.0, dt_pow=4)
         for N in (32, 64, 128)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(rates > 3.6), rates


def test_burgers_at_seeded_converges_second_order():
    """Fig. 2 (green line): WS + AT keeps slope -2 under delays."""
    for order in (2, 4):
        e = [_conv_run(N, order, P=8, L=3, mode=oracle.SEEDED, T=0.5, nu=0.1, lam=1.0) for N in (64, 128, 256)]
        rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        assert np.all(rates > 1.7), (order, rates)


def test_fig2_linear_advection_diffusion_three_configurations():
    """Fig. 2, P = 8: synchronous + standard and WS + AT converge at slope -2;
    WS + standard schemes (delayed halo used as is) lose accuracy."""
    nu, c, kappa, T = 0.1, 1.0, 2, 0.5

    def err(N, mode, at_w):
        x, dx = W.grid(N)
        dt0 = 1.0 * dx * dx
        n = int(math.ceil(T / dt0))
        dt = T / n
        u, _ = oracle.run(np.sin(kappa * x), P=8, order=2, L=3, nu=nu, dt=dt, n_steps=n, eq=oracle.EQ_LINEAR,
                          adv_c=c, delay_mode=mode, seed=9, at_weights=at_w)
        exact = np.exp(-nu * kappa ** 2 * T) * np.sin(kappa * (x - c * T))
        return np.mean(np.abs(u - exact))

    Ns = (64, 128, 256)
    ts = [err(N, oracle.SYNC, True) for N in Ns]
    at = [err(N, oracle.SEEDED, True) for N in Ns]
    st = [err(N, oracle.SEEDED, False) for N in Ns]
    r_ts = np.log2(ts[0] / ts[-1]) / 2
    r_at = np.log2(at[0] / at[-1]) / 2
    r_st = np.log2(st[0] / st[-1]) / 2
    assert 1.8 < r_ts < 2.3 and 1.7 < r_at < 2.4, (r_ts, r_at)
    assert r_st < 1.2, r_st
    assert st[-1] > 10 * at[-1]


def _tanh_exact(x, t, nu, a, c, xc):
    return c - a * np.tanh(a * (x - xc - c * t) / (2 * nu))


def test_tanh_travelling_wave_converges():
    """Closed-form viscous-Burgers travelling wave with exact ghost values at
    the two ends of [-pi, pi): slope -2 synchronous and with seeded AT delays."""
    nu, a, c, T = 0.2, 0.5, 0.3, 0.5

    def err(N, mode):
        x, dx = W.grid(N, x0=-math.pi)
        dt0 = 1.0 * dx * dx
        n = int(math.ceil(T / dt0))
        dt = T / n
        u0 = _tanh_exact(x, 0.0, nu, a, c, 0.0)
        u, _ = oracle.run(u0, P=8, order=2, L=2, nu=nu, dt=dt, n_steps=n, x0=-math.pi, dx=dx,
                          bc=oracle.BC_TANH, tanh=(a, c, 0.0), delay_mode=mode, seed=4)
        return np.mean(np.abs(u - _tanh_exact(x, T, nu, a, c, 0.0)))

    for mode in (oracle.SYNC, oracle.SEEDED):
        e = [err(N, mode) for N in (64, 128, 256)]
        rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        assert np.all(rates > 1.7), (mode, rates)


# --------------------------------------------------------------------------
# Error scaling law, Eq. err_scaling: <E> ~ (P/N) dx^2 (<k^2> + <k>)
# --------------------------------------------------------------------------
def _async_error(N, P, k_const, n_steps=400):
    x, dx = W.grid(N)
    u0 = W.u0_two_modes(N)
    nu = 0.05
    dt = W.dt_rule(u0, dx, nu)
    us, _ = oracle.run(u0, P=P, order=2, L=3, nu=nu, dt=dt, n_steps=n_steps)
    rep = np.full((n_steps, P, 2), k_const, np.int8)
    ua, _ = oracle.run(u0, P=P, order=2, L=3, nu=nu, dt=dt, n_steps=n_steps,
                       delay_mode=oracle.REPLAY, replay=rep)
    return np.mean(np.abs(ua - us))


def test_error_grows_linearly_with_P():
    e8, e16, e32 = (_async_error(512, P, 2) for P in (8, 16, 32))
    assert 1.6 < e16 / e8 < 2.5 and 1.6 < e32 / e16 < 2.5, (e8, e16, e32)


def test_error_grows_with_delay_moments():
    """Constant delay k: <k^2> + <k> = 2, 6, 12 for k = 1, 2, 3."""
    e1, e2, e3 = (_async_error(512, 16, k) for k in (1, 2, 3))
    assert e1 < e2 < e3
    assert 2.0 < e2 / e1 < 4.5 and 1.5 < e3 / e2 < 2.6, (e1, e2, e3)


# --------------------------------------------------------------------------
# Window runs (used to sample full-size results one subdomain at a time)
# --------------------------------------------------------------------------
def test_window_run_matches_full_run_in_its_centre():
    N, P, n = 2048, 64, 30
    u0 = W.u0_fourier(N, modes=16, seed=2)
    x, dx = W.grid(N)
    kw = dict(N=N, P=P, order=4, L=3, nu=1e-3, dt=1e-6, n_steps=n, forcing_amp=0.1,
              delay_mode=oracle.SEEDED, seed=3)
    full, _ = oracle.run(u0, **kw)
    M = N // P
    p_lo, p_count = 20, 5         # 5 subdomains; R n = 60 < 2 M points of margin
    win, _ = oracle.run(u0[p_lo * M:(p_lo + p_count) * M], p_lo=p_lo, p_count=p_count, **kw)
    mid = slice(2 * M, 3 * M)
    assert np.array_equal(win[mid], full[(p_lo + 2) * M:(p_lo + 3) * M])


def test_window_run_wraps_around_the_domain_end():
    """A window that runs past subdomain P-1 continues at subdomain 0."""
    N, P, n = 1024, 32, 20
    u0 = W.u0_fourier(N, modes=16, seed=5)
    kw = dict(N=N, P=P, order=2, L=2, nu=1e-2, dt=1e-5, n_steps=n, forcing_amp=0.1,
              delay_mode=oracle.SEEDED, seed=8)
    full, _ = oracle.run(u0, **kw)
    M = N // P
    p_lo, p_count = P - 2, 5     # subdomains P-2, P-1, 0, 1, 2
    idx = np.concatenate([np.arange((P - 2) * M, N), np.arange(0, 3 * M)])
    win, _ = oracle.run(u0[idx], p_lo=p_lo, p_count=p_count, **kw)
    assert np.array_equal(win[2 * M:3 * M], full[0:M])
