"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and
the benchmark.

This module holds no arithmetic of the method itself (no stencil, no delay
rule, no time update): only grids, initial fields, the time-step rule that
turns a configuration into a dt, and the named workload configurations.

Workloads (1D viscous Burgers on the periodic interval [0, 2 pi)):

* ``burgers1d_n4096``: N = 4096 points, P = 16 subdomains, order 2, L = 2,
  nu = 0.02, u0 = sin(x) + 0.5 sin(3x + 1), FP64, seeded delays (seed 1),
  1000 steps.
* ``burgers1d_forced_n2p26``: N = 2^26, P = 65536 subdomains of 1024 points,
  order 4, L = 3, nu = 1e-3, forcing A sin(x) with A = 0.1,
  u0 = sum_{k=1}^{64} k^-1 sin(k x + phi_k), phi_k ~ U[0, 2 pi) (seed 2),
  seeded delays (seed 3) or free-running delays, 10^4 steps, FP32 or FP64.
* ``burgers1d_ensemble_2048``: 2048 independent 1D problems on [-pi, pi),
  N_j = 2^x_j (x_j ~ U[10, 16]) rounded to a multiple of 256 (P_j = N_j / 256
  subdomains of M = 256 points), nu_j log-uniform in [1e-3, 1e-1], delay bound
  L_j ~ U{1, 2, 3}, order 2, FP32, 5000 steps; initial data and boundary
  values from the travelling tanh wave u = c - a tanh(a (x - xc - c t)/(2 nu))
  with c_j ~ U[-0.5, 0.5], a_j = min(0.5, 0.5 nu_j / dx_j) (a front at least
  4 dx wide), xc = 0; seed 6.

* ``burgers1d_adjoint_n2p20``: see ``adjoint_workload``.
* ``burgers3d_n512``: see ``u0_spectral3d``.

The paper's own runs (3D Burgers' turbulence from a multi-scale sinusoidal
initial condition, Sec. 3.1) use no dataset; these fields stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def grid(N: int, length: float = TWO_PI, x0: float = 0.0):
    """Cell positions x_i = x0 + i dx, i = 0..N-1, and dx = length / N."""
    dx = length / N
    return x0 + np.arange(N, dtype=np.float64) * dx, dx


def u0_two_modes(N: int) -> np.ndarray:
    """u0 = sin(x) + 0.5 sin(3x + 1) on [0, 2 pi)."""
    x, _ = grid(N)
    return np.sin(x) + 0.5 * np.sin(3.0 * x + 1.0)


def u0_fourier(N: int, modes: int = 64, seed: int = 2) -> np.ndarray:
    """u0 = sum_{k=1}^{modes} k^-1 sin(k x + phi_k), phi_k ~ U[0, 2 pi).

    Evaluated through an inverse real FFT (exact up to rounding), so that
    N = 2^26 takes seconds rather than minutes.
    """
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, TWO_PI, size=modes)
    if N < 2 * modes + 2:
        x, _ = grid(N)
        k = np.arange(1, modes + 1)
        return (np.sin(np.outer(x, k) + phi) / k).sum(axis=1)
    X = np.zeros(N // 2 + 1, dtype=np.complex128)
    k = np.arange(1, modes + 1)
    # a sin(kx + phi) = Re(-i a e^{i phi} e^{ikx}); irfft divides by N and
    # doubles the positive frequencies.
    X[1:modes + 1] = (N / 2.0) * (-1j) * np.exp(1j * phi) / k
    return np.fft.irfft(X, n=N)


def dt_rule(u0: np.ndarray, dx: float, nu: float, dim: int = 1, cfl: float = 0.2) -> float:
    """dt = cfl * min(dx / max|u0|, dx^2 / (2 dim nu)): the tighter of the
    advective and the diffusive limit, scaled by the CFL number."""
    umax = float(np.max(np.abs(u0)))
    lim = []
    if umax > 0.0:
        lim.append(dx / umax)
    if nu > 0.0:
        lim.append(dx * dx / (2.0 * dim * nu))
    return cfl * min(lim)


def config(name: str) -> dict:
    """Parameters of a named workload (initial field generated on demand)."""
    if name == "burgers1d_n4096":
        return dict(name=name, N=4096, P=16, order=2, L=2, nu=0.02, forcing_amp=0.0,
                    u0=("two_modes",), seed=1, n_steps=1000, dtype="f64")
    if name == "burgers1d_forced_n2p26":
        return dict(name=name, N=1 << 26, P=65536, order=4, L=3, nu=1e-3, forcing_amp=0.1,
                    u0=("fourier", 64, 2), seed=3, n_steps=10000, dtype="f32")
    raise KeyError(name)


def initial_field(cfg: dict, N: int | None = None) -> np.ndarray:
    N = cfg["N"] if N is None else N
    kind = cfg["u0"]
    if kind[0] == "two_modes":
        return u0_two_modes(N)
    if kind[0] == "fourier":
        return u0_fourier(N, modes=kind[1], seed=kind[2])
    raise KeyError(kind)


def ensemble(n_inst: int = 2048, seed: int = 6, M: int = 256, log2_n=(10.0, 16.0), nu_range=(1e-3, 1e-1),
             L_choices=(1, 2, 3), cfl: float = 0.2) -> list:
    """Instances of an ensemble of travelling-wave problems (see the module
    docstring): a list of dicts with n, L, nu, dt, length, origin, tanh_a,
    tanh_c, tanh_xc and seed (the instance's seeded-delay seed).  dt follows
    ``dt_rule`` on the instance's initial field."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        n = int(round(2.0 ** rng.uniform(*log2_n) / M)) * M
        n = max(n, M)
        nu = float(np.exp(rng.uniform(math.log(nu_range[0]), math.log(nu_range[1]))))
        L = int(rng.choice(L_choices))
        c = float(rng.uniform(-0.5, 0.5))
        dx = TWO_PI / n
        a = min(0.5, 0.5 * nu / dx)
        inst = dict(n=n, L=L, nu=nu, length=TWO_PI, origin=-math.pi, tanh_a=a, tanh_c=c, tanh_xc=0.0,
                    seed=int(rng.integers(0, 2**62)))
        inst["dt"] = dt_rule(tanh_wave(inst, 0.0), dx, nu, cfl=cfl)
        out.append(inst)
    return out


def tanh_wave(inst: dict, t: float) -> np.ndarray:
    """The instance's travelling wave u = c - a tanh(a (x - xc - c t)/(2 nu))
    at time t on its grid x_i = origin + i length / n."""
    x, _ = grid(inst["n"], inst["length"], inst["origin"])
    a, c = inst["tanh_a"], inst["tanh_c"]
    return c - a * np.tanh(a * (x - inst["tanh_xc"] - c * t) / (2.0 * inst["nu"]))


def instance_field(inst: dict) -> np.ndarray:
    """Initial field of an instance: its own ``u0`` if it has one, else the
    travelling wave at t = 0."""
    if "u0" in inst:
        return np.asarray(inst["u0"], dtype=np.float64)
    return tanh_wave(inst, 0.0)


def ensemble_field(instances: list) -> np.ndarray:
    """Initial state of an ensemble: the instances' fields at t = 0, end to end."""
    return np.concatenate([instance_field(d) for d in instances])


def adjoint_workload(N: int = 1 << 20, M: int = 1024) -> dict:
    """The adjoint workload ``burgers1d_adjoint_n2p20``: N = 2^20 points in
    subdomains of M = 1024 (P = 1024), order 2, L = 2, nu = 0.01, seeded
    delays (seed 7), 2000 steps, checkpoints every 100; u0 = sin x +
    0.5 sin(3x + 1); the target is the run (same delays) from u0 + 0.01 q
    with viscosity 1.05 nu, q an 8-mode field with seeded amplitudes and
    phases (seed 7), normalised to max |q| = 1.  Loss ||u(T) - u_target||^2."""
    x, dx = grid(N)
    u0 = u0_two_modes(N)
    rng = np.random.default_rng(7)
    amp = rng.uniform(0.5, 1.0, size=8)
    phi = rng.uniform(0.0, TWO_PI, size=8)
    q = sum(amp[k] * np.sin((k + 1) * x + phi[k]) for k in range(8))
    q /= np.max(np.abs(q))
    nu = 0.01
    return dict(name="burgers1d_adjoint_n2p20", N=N, P=N // M, order=2, L=2, nu=nu, seed=7, n_steps=2000,
                interval=100, u0=u0, u0_target=u0 + 0.01 * q, nu_target=1.05 * nu, dt=dt_rule(u0, dx, nu))


def u0_spectral3d(n: int, seed: int = 4, kmax: int = 32) -> np.ndarray:
    """Periodic n^3 field (shape (n, n, n), x fastest) with energy spectrum
    E(k) ~ k^-5/3 for 1 <= |k| <= kmax: every wavevector in that shell gets
    amplitude |k|^-11/6 and a uniform random phase (seeded), the real field is
    the inverse real FFT, normalised to max |u0| = 1 (the workload
    ``burgers3d_n512``: n = 512, nu = 5e-3, subdomains of 32^3, order 2, L = 2,
    seed 4, 2000 steps)."""
    rng = np.random.default_rng(seed)
    km = min(kmax, n // 2 - 1)
    k1 = np.arange(-km, km + 1)
    kz = np.arange(0, km + 1)
    KX, KY, KZ = np.meshgrid(k1, k1, kz, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    amp = np.where((kk >= 1) & (kk <= kmax), np.power(np.maximum(kk, 1.0), -11.0 / 6.0), 0.0)
    phase = rng.uniform(0.0, TWO_PI, size=amp.shape)
    X = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    X[np.ix_(k1 % n, k1 % n, kz)] = amp * np.exp(1j * phase)
    u = np.fft.irfftn(X, s=(n, n, n), axes=(0, 1, 2))
    return u / np.max(np.abs(u))


def random_delays(n_steps: int, P: int, L: int, seed: int, faces: int = 2) -> np.ndarray:
    """Uniform delays in {0..L}, shape [n_steps, P, faces], int8 (for replay)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, L + 1, size=(n_steps, P, faces), dtype=np.int8)
