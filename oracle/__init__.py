"""CPU oracle for the weakly-synchronous AT method of arXiv 1911.05769.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg (``bench.py``) may import this package.  It shares
no code with the CUDA library in ``paper_1911_05769_gb300``; the two are
compared element by element.

The arithmetic lives in ``at_oracle.c`` (plain FP64 C, compiled with
``-O2 -ffp-contract=off``).  This module compiles it on first use and marshals
numpy arrays through ctypes.

Sections followed (see the C file for the details): Eq. BS (Burgers), Sec. 3.2
(forward Euler, central differences, AT schemes at process-boundary points),
Eq. AT1 / Eq. AT2 (AT coefficients), Sec. 5.2 and Algorithm 2 (split form:
halo approximation, then the unchanged stencil; synchrony during start-up).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "at_oracle.c")
_LIB = os.path.join(_HERE, "libat_oracle.so")
_lock = threading.Lock()
_lib = None

SYNC, SEEDED, REPLAY = 0, 1, 2
EQ_BURGERS, EQ_LINEAR = 0, 1
BC_PERIODIC, BC_TANH = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libat_oracle.so`` (plain gcc, with
    OpenMP over subdomains where the compiler has it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-shared", "-fPIC"]
        try:
            subprocess.check_call(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + [_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64), ("P", ctypes.c_int64),
        ("p_lo", ctypes.c_int64), ("p_count", ctypes.c_int64),
        ("order", ctypes.c_int32), ("L", ctypes.c_int32),
        ("nu", ctypes.c_double), ("dt", ctypes.c_double),
        ("x0", ctypes.c_double), ("dx", ctypes.c_double),
        ("forcing_amp", ctypes.c_double),
        ("eq", ctypes.c_int32), ("bc", ctypes.c_int32),
        ("adv_c", ctypes.c_double),
        ("tanh_a", ctypes.c_double), ("tanh_c", ctypes.c_double), ("tanh_xc", ctypes.c_double),
        ("delay_mode", ctypes.c_int32), ("per_subdomain", ctypes.c_int32),
        ("at_weights", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


class Cfg3(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64 * 3), ("P", ctypes.c_int64 * 3), ("L", ctypes.c_int32), ("delay_mode", ctypes.c_int32),
        ("nu", ctypes.c_double), ("dt", ctypes.c_double), ("dx", ctypes.c_double * 3), ("seed", ctypes.c_uint64),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.at_oracle_splitmix64.restype = ctypes.c_uint64
            L.at_oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.at_oracle_seeded_delay.restype = ctypes.c_int
            L.at_oracle_seeded_delay.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.at_oracle_weights.restype = ctypes.c_int
            L.at_oracle_weights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_double)]
            L.at_oracle_extrapolate.restype = ctypes.c_double
            L.at_oracle_extrapolate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_double)]
            L.at_oracle_derivs.restype = ctypes.c_int
            L.at_oracle_derivs.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.at_oracle_run.restype = ctypes.c_int
            L.at_oracle_run.argtypes = [ctypes.POINTER(Cfg), ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.at_oracle_adjoint.restype = ctypes.c_int
            L.at_oracle_adjoint.argtypes = [ctypes.POINTER(Cfg), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_double)]
            L.at_oracle_run3d.restype = ctypes.c_int
            L.at_oracle_run3d.argtypes = [ctypes.POINTER(Cfg3), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]
            L.at_oracle_run3d_system.restype = ctypes.c_int
            L.at_oracle_run3d_system.argtypes = [ctypes.POINTER(Cfg3), ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.at_oracle_threads.restype = ctypes.c_int
            L.at_oracle_threads.argtypes = [ctypes.c_int]
            L.at_oracle_cfg3_size.restype = ctypes.c_int64
            if L.at_oracle_cfg3_size() != ctypes.sizeof(Cfg3):
                raise RuntimeError("oracle: 3D configuration struct layout mismatch")
            L.at_oracle_cfg_size.restype = ctypes.c_int64
            if L.at_oracle_cfg_size() != ctypes.sizeof(Cfg):
                raise RuntimeError("oracle: configuration struct layout mismatch")
            _lib = L
    return _lib


def threads(n: int = 0) -> int:
    """Sets the oracle's thread count (n > 0) and returns the count in force.
    Results do not depend on it: the threads share out whole subdomains (1D)
    or planes (3D), and every point is computed by the same arithmetic."""
    return int(lib().at_oracle_threads(int(n)))


def _dptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def splitmix64(seed: int, i: int) -> int:
    return int(lib().at_oracle_splitmix64(seed & (2**64 - 1), i & (2**64 - 1)))


def seeded_delay(seed, n, p, P, face, F, L) -> int:
    return int(lib().at_oracle_seeded_delay(seed, n, p, P, face, F, L))


def weights(s: int, k: int, at_weights: bool = True) -> np.ndarray:
    w = np.zeros(s, dtype=np.float64)
    rc = lib().at_oracle_weights(s, k, int(at_weights), w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError(f"oracle weights: rc={rc}")
    return w


def extrapolate(s: int, k: int, levels, at_weights: bool = True) -> float:
    lev = np.ascontiguousarray(levels, dtype=np.float64)
    return float(lib().at_oracle_extrapolate(s, k, int(at_weights),
                                             lev.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def derivs(order: int, v, dx: float):
    v = np.ascontiguousarray(v, dtype=np.float64)
    d1, d2 = ctypes.c_double(), ctypes.c_double()
    rc = lib().at_oracle_derivs(order, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), dx,
                                ctypes.byref(d1), ctypes.byref(d2))
    if rc != 0:
        raise ValueError("oracle derivs: bad order")
    return d1.value, d2.value


def run(u0, *, N=None, P, order, L, nu, dt, n_steps, x0=0.0, dx=None, length=2 * np.pi,
        forcing_amp=0.0, eq=EQ_BURGERS, adv_c=0.0, bc=BC_PERIODIC, tanh=(0.0, 0.0, 0.0),
        delay_mode=SYNC, seed=0, replay=None, per_subdomain=False, at_weights=True,
        p_lo=0, p_count=None, want_k=False):
    """Advance ``u0`` by ``n_steps`` forward-Euler steps of the AT method.

    ``u0`` holds the field of subdomains ``p_lo .. p_lo+p_count-1`` (the whole
    domain by default).  Returns ``(u, hist)`` or ``(u, hist, k_used)``.
    """
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    if N is None:
        N = u0.size
    if p_count is None:
        p_count = P
    if dx is None:
        dx = length / N
    c = Cfg(N=N, P=P, p_lo=p_lo, p_count=p_count, order=order, L=L, nu=nu, dt=dt, x0=x0, dx=dx,
            forcing_amp=forcing_amp, eq=eq, bc=bc, adv_c=adv_c, tanh_a=tanh[0], tanh_c=tanh[1],
            tanh_xc=tanh[2], delay_mode=delay_mode, per_subdomain=int(per_subdomain),
            at_weights=int(at_weights), pad_=0, seed=seed & (2**64 - 1))
    W = p_count * (N // P)
    if u0.size != W:
        raise ValueError(f"oracle run: u0 has {u0.size} values, window needs {W}")
    out = np.empty(W, dtype=np.float64)
    hist = np.zeros(L + 1, dtype=np.int64)
    rep = None
    if delay_mode == REPLAY:
        rep = np.ascontiguousarray(replay, dtype=np.int8)
        if rep.size != n_steps * p_count * 2:
            raise ValueError("oracle run: replay array has the wrong size")
    kk = np.empty((n_steps, p_count, 2), dtype=np.int8) if want_k else None
    rc = lib().at_oracle_run(ctypes.byref(c), n_steps, _dptr(rep), _dptr(u0), _dptr(out),
                             _dptr(hist), _dptr(kk))
    if rc != 0:
        raise ValueError(f"oracle run failed: rc={rc}")
    return (out, hist, kk) if want_k else (out, hist)


def adjoint(u0, lam_T, *, N=None, P, order, L, nu, dt, n_steps, x0=0.0, dx=None, length=2 * np.pi,
            forcing_amp=0.0, delay_mode=SYNC, seed=0, replay=None, per_subdomain=False, at_weights=True):
    """Discrete adjoint of ``run`` (Burgers, whole periodic domain).

    Returns ``(u_T, lam_0, dnu)``: the run's final level, dJ/du^0 and dJ/dnu
    for a J whose gradient with respect to u^{n_steps} is ``lam_T``.
    """
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    lam_T = np.ascontiguousarray(lam_T, dtype=np.float64)
    if N is None:
        N = u0.size
    if dx is None:
        dx = length / N
    c = Cfg(N=N, P=P, p_lo=0, p_count=P, order=order, L=L, nu=nu, dt=dt, x0=x0, dx=dx,
            forcing_amp=forcing_amp, eq=EQ_BURGERS, bc=BC_PERIODIC, adv_c=0.0, tanh_a=0.0, tanh_c=0.0,
            tanh_xc=0.0, delay_mode=delay_mode, per_subdomain=int(per_subdomain), at_weights=int(at_weights),
            pad_=0, seed=seed & (2**64 - 1))
    if u0.size != N or lam_T.size != N:
        raise ValueError("oracle adjoint: u0 and lam_T need N values")
    rep = None
    if delay_mode == REPLAY:
        rep = np.ascontiguousarray(replay, dtype=np.int8)
        if rep.size != n_steps * P * 2:
            raise ValueError("oracle adjoint: replay array has the wrong size")
    u_T = np.empty(N, dtype=np.float64)
    lam_0 = np.empty(N, dtype=np.float64)
    dnu = ctypes.c_double()
    rc = lib().at_oracle_adjoint(ctypes.byref(c), n_steps, _dptr(rep), _dptr(u0), _dptr(lam_T), _dptr(u_T),
                                 _dptr(lam_0), ctypes.byref(dnu))
    if rc != 0:
        raise ValueError(f"oracle adjoint failed: rc={rc}")
    return u_T, lam_0, dnu.value


def run3d(u0, *, P, L, nu, dt, n_steps, dx=None, length=2 * np.pi, delay_mode=SYNC, seed=0, replay=None):
    """3D AT run (order 2, six faces per subdomain) of ``u0`` shaped
    (n2, n1, n0) (x fastest) with P = (P0, P1, P2) subdomains per axis.
    Returns ``(u, hist)`` with u of the same shape."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    n2, n1, n0 = u0.shape
    if dx is None:
        dx = (length / n0, length / n1, length / n2)
    c = Cfg3()
    c.n[0], c.n[1], c.n[2] = n0, n1, n2
    c.P[0], c.P[1], c.P[2] = P
    c.L, c.delay_mode, c.nu, c.dt = L, delay_mode, nu, dt
    c.dx[0], c.dx[1], c.dx[2] = dx
    c.seed = seed & (2**64 - 1)
    NP = P[0] * P[1] * P[2]
    rep = None
    if delay_mode == REPLAY:
        rep = np.ascontiguousarray(replay, dtype=np.int8)
        if rep.size != n_steps * NP * 6:
            raise ValueError("oracle run3d: replay array has the wrong size")
    out = np.empty_like(u0)
    hist = np.zeros(L + 1, dtype=np.int64)
    rc = lib().at_oracle_run3d(ctypes.byref(c), n_steps, _dptr(rep), _dptr(u0), _dptr(out), _dptr(hist))
    if rc != 0:
        raise ValueError(f"oracle run3d failed: rc={rc}")
    return out, hist


def run3d_system(q0, *, kappa, P, L, dt, n_steps, dx=None, length=2 * np.pi, delay_mode=SYNC, seed=0, replay=None):
    """The system of Eq. BS in 3D: q0 shaped (nf, n2, n1, n0) with the velocity
    components in fields 0, 1, 2 and passive scalars after them; kappa[f] the
    viscosity (velocity) or diffusivity (scalars) of field f.  Same grid,
    subdomains, delays and AT halos as ``run3d``.  Returns ``(q, hist)``."""
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    nf, n2, n1, n0 = q0.shape
    kap = np.ascontiguousarray(kappa, dtype=np.float64)
    if kap.size != nf:
        raise ValueError("run3d_system: one kappa per field")
    if dx is None:
        dx = (length / n0, length / n1, length / n2)
    c = Cfg3()
    c.n[0], c.n[1], c.n[2] = n0, n1, n2
    c.P[0], c.P[1], c.P[2] = P
    c.L, c.delay_mode, c.nu, c.dt = L, delay_mode, 0.0, dt
    c.dx[0], c.dx[1], c.dx[2] = dx
    c.seed = seed & (2**64 - 1)
    NP = P[0] * P[1] * P[2]
    rep = None
    if delay_mode == REPLAY:
        rep = np.ascontiguousarray(replay, dtype=np.int8)
        if rep.size != n_steps * NP * 6:
            raise ValueError("run3d_system: replay array has the wrong size")
    out = np.empty_like(q0)
    hist = np.zeros(L + 1, dtype=np.int64)
    rc = lib().at_oracle_run3d_system(ctypes.byref(c), nf, _dptr(kap), n_steps, _dptr(rep), _dptr(q0), _dptr(out),
                                      _dptr(hist))
    if rc != 0:
        raise ValueError(f"oracle run3d_system failed: rc={rc}")
    return out, hist
