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


def random_delays(n_steps: int, P: int, L: int, seed: int, faces: int = 2) -> np.ndarray:
    """Uniform delays in {0..L}, shape [n_steps, P, faces], int8 (for replay)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, L + 1, size=(n_steps, P, faces), dtype=np.int8)
