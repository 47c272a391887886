"""ctypes binding of the C ABI in ``include/at.h`` -- argument marshalling only.

Every function has the name and the argument order of its C counterpart and
returns the C return code.  Pointers are plain integers (device or host
addresses, e.g. ``tensor.data_ptr()``).  The library is loaded on first use;
if ``libat.so`` has not been built, the first call raises ``RuntimeError``
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libat.so")
_lock = threading.Lock()
_lib = None

AT_OK = 0
AT_ERR_ARG = -1
AT_ERR_UNSTABLE = -2
AT_ERR_RESIDENCY = -3
AT_ERR_CUDA = -4
AT_ERR_TIMEOUT = -5
AT_ERR_STATE = -6

AT_F64 = 0
AT_F32 = 1
AT_BC_PERIODIC = 0
AT_BC_EXACT_TANH = 1

AT_SYNC = 0
AT_SEEDED = 1
AT_FREE = 2
AT_REPLAY = 3

AT_FLAG_PER_SUBDOMAIN_DELAY = 1
AT_FLAG_ALLOW_UNSTABLE = 2
AT_FLAG_TEST_SKIP_PUBLISH = 4
AT_FLAG_VISCOUS_FP64 = 8
AT_FLAG_VISCOUS_FP32 = 16
AT_FLAG_COMPENSATED = 32

AT_NOALLOC_SCRATCH_BYTES = 8 * 1024 * 1024


class at_grid(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("bc", ctypes.c_int32), ("dtype", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("n", ctypes.c_int64 * 3), ("length", ctypes.c_double * 3), ("origin", ctypes.c_double * 3),
        ("forcing_amp", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t), ("stream", ctypes.c_void_p),
        ("timeout_ns", ctypes.c_int64), ("max_ctas", ctypes.c_int32), ("stages", ctypes.c_int32),
        ("test_skip_step", ctypes.c_int64), ("steps_per_pass", ctypes.c_int32), ("tile_subdomains", ctypes.c_int32),
        ("sub", ctypes.c_int64 * 3),
    ]


class at_info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64), ("P", ctypes.c_int64), ("M", ctypes.c_int64),
        ("order", ctypes.c_int32), ("L", ctypes.c_int32), ("R", ctypes.c_int32), ("s", ctypes.c_int32),
        ("T", ctypes.c_int32), ("ctas", ctypes.c_int32), ("threads", ctypes.c_int32), ("stages", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int64), ("step", ctypes.c_int64), ("sm_count", ctypes.c_int32),
        ("dtype", ctypes.c_int32), ("steps_per_pass", ctypes.c_int32), ("viscous_fp64", ctypes.c_int32),
        ("tile_subdomains", ctypes.c_int32),
    ]


class at_instance(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("L", ctypes.c_int32), ("bc", ctypes.c_int32),
        ("length", ctypes.c_double), ("origin", ctypes.c_double), ("nu", ctypes.c_double), ("dt", ctypes.c_double),
        ("tanh_a", ctypes.c_double), ("tanh_c", ctypes.c_double), ("tanh_xc", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class at_tune_result(ctypes.Structure):
    _fields_ = [
        ("ctas", ctypes.c_int32), ("stages", ctypes.c_int32), ("steps_per_pass", ctypes.c_int32),
        ("n_tried", ctypes.c_int32), ("best_ms", ctypes.c_double), ("first_ms", ctypes.c_double),
        ("tile_subdomains", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


# (name, restype, argtypes) of every exported entry point
_SIGNATURES = [
    ("at_workspace_bytes", ctypes.c_size_t,
     [ctypes.POINTER(at_grid), ctypes.c_int64, ctypes.c_int, ctypes.c_int]),
    ("at_create", ctypes.c_int,
     [ctypes.POINTER(at_grid), ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
      ctypes.POINTER(ctypes.c_void_p)]),
    ("at_set_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("at_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]),
    ("at_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("at_state_error", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("at_fma_peak", ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    ("at_status", ctypes.c_int, [ctypes.c_void_p]),
    ("at_delay_stats", ctypes.c_int,
     [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
      ctypes.POINTER(ctypes.c_double)]),
    ("at_get_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(at_info)]),
    ("at_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("at_last_error", ctypes.c_char_p, []),
    ("at_step_noalloc", ctypes.c_int,
     [ctypes.POINTER(at_grid), ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
      ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]),
    ("at_batch_workspace_bytes", ctypes.c_size_t,
     [ctypes.POINTER(at_grid), ctypes.c_int64, ctypes.POINTER(at_instance), ctypes.c_int64, ctypes.c_int]),
    ("at_create_batch", ctypes.c_int,
     [ctypes.POINTER(at_grid), ctypes.c_int64, ctypes.POINTER(at_instance), ctypes.c_int64, ctypes.c_int,
      ctypes.POINTER(ctypes.c_void_p)]),
    ("at_tune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(at_tune_result)]),
    ("at_system_workspace_bytes", ctypes.c_size_t,
     [ctypes.POINTER(at_grid), ctypes.c_int64, ctypes.c_int, ctypes.c_int]),
    ("at_create_system", ctypes.c_int,
     [ctypes.POINTER(at_grid), ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
      ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    ("at_moments", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("at_step_levels", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    ("at_set_history", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]),
    ("at_checkpoint_bytes", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]),
    ("at_step_checkpointed", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    ("at_adjoint_workspace_bytes", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64]),
    ("at_adjoint", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
]

EXPORTED = [s[0] for s in _SIGNATURES]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"CUDA library {_LIB_PATH} is missing: run "
                                   "`python -m paper_1911_05769_gb300.build` (no CPU fallback exists)")
            L = ctypes.CDLL(_LIB_PATH)
            for name, res, args in _SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class AtError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed with {code}: {at_last_error()}")
        self.code = code


def at_workspace_bytes(grid: at_grid, P: int, scheme_order: int, L: int) -> int:
    return int(lib().at_workspace_bytes(ctypes.byref(grid), P, scheme_order, L))


def at_create(grid: at_grid, P: int, scheme_order: int, L: int, nu: float, dt: float):
    """Returns (code, handle)."""
    h = ctypes.c_void_p()
    rc = lib().at_create(ctypes.byref(grid), P, scheme_order, L, nu, dt, ctypes.byref(h))
    return rc, h


def at_set_state(h, u_ptr: int) -> int:
    return lib().at_set_state(h, ctypes.c_void_p(u_ptr))


def at_step(h, n_steps: int, delay_mode: int, delays_ptr: int | None = None) -> int:
    return lib().at_step(h, n_steps, delay_mode, ctypes.c_void_p(delays_ptr) if delays_ptr else None)


def at_state(h, dst_ptr: int) -> int:
    return lib().at_state(h, ctypes.c_void_p(dst_ptr))


def at_state_error(h, dst_ptr: int) -> int:
    return lib().at_state_error(h, ctypes.c_void_p(dst_ptr))


def at_fma_peak(dtype: int, trips: int) -> float:
    """FMAs per second of the current GPU for AT_F64 / AT_F32 (raises on error)."""
    out = ctypes.c_double()
    rc = lib().at_fma_peak(dtype, trips, ctypes.byref(out))
    if rc != AT_OK:
        raise AtError(rc, "at_fma_peak")
    return out.value


def at_status(h) -> int:
    return lib().at_status(h)


def at_delay_stats(h, L: int):
    """Returns (code, hist[L+1] list, mean_k, mean_k2)."""
    hist = (ctypes.c_int64 * (L + 1))()
    m1, m2 = ctypes.c_double(), ctypes.c_double()
    rc = lib().at_delay_stats(h, hist, ctypes.byref(m1), ctypes.byref(m2))
    return rc, list(hist), m1.value, m2.value


def at_get_info(h):
    info = at_info()
    rc = lib().at_get_info(h, ctypes.byref(info))
    return rc, info


def at_destroy(h) -> int:
    return lib().at_destroy(h)


def at_step_noalloc(grid: at_grid, P: int, scheme_order: int, L: int, nu: float, dt: float, u_ptr: int,
                    n_steps: int, delay_mode: int, delays_ptr: int | None = None) -> int:
    """Allocation-free run for callers that cannot allocate device memory: the
    state at ``u_ptr`` (device) is advanced in place; scratch is the library's
    fixed array (see include/at.h).  Synchronises and returns the status."""
    return lib().at_step_noalloc(ctypes.byref(grid), P, scheme_order, L, nu, dt, ctypes.c_void_p(u_ptr), n_steps,
                                 delay_mode, ctypes.c_void_p(delays_ptr) if delays_ptr else None)


def at_batch_workspace_bytes(grid: at_grid, instances, M: int, scheme_order: int) -> int:
    """instances: ctypes array of at_instance."""
    return int(lib().at_batch_workspace_bytes(ctypes.byref(grid), len(instances), instances, M, scheme_order))


def at_create_batch(grid: at_grid, instances, M: int, scheme_order: int):
    """Returns (code, handle).  instances: ctypes array of at_instance."""
    h = ctypes.c_void_p()
    rc = lib().at_create_batch(ctypes.byref(grid), len(instances), instances, M, scheme_order, ctypes.byref(h))
    return rc, h


def at_tune(h, n_steps: int, delay_mode: int):
    """Returns (code, at_tune_result)."""
    res = at_tune_result()
    rc = lib().at_tune(h, n_steps, delay_mode, ctypes.byref(res))
    return rc, res


def at_system_workspace_bytes(grid: at_grid, P: int, L: int, nfields: int) -> int:
    return int(lib().at_system_workspace_bytes(ctypes.byref(grid), P, L, nfields))


def at_create_system(grid: at_grid, P: int, L: int, kappa, dt: float):
    """Returns (code, handle); kappa: one viscosity/diffusivity per field (3..5 fields)."""
    kap = (ctypes.c_double * len(kappa))(*kappa)
    h = ctypes.c_void_p()
    rc = lib().at_create_system(ctypes.byref(grid), P, L, len(kappa), kap, dt, ctypes.byref(h))
    return rc, h


def at_moments(h, nfields: int):
    """Returns (code, [(mean, mean square) per field])."""
    out = (ctypes.c_double * (2 * nfields))()
    rc = lib().at_moments(h, out)
    return rc, [(out[2 * f], out[2 * f + 1]) for f in range(nfields)]


def _vp(ptr):
    return ctypes.c_void_p(ptr) if ptr else None


def at_step_levels(h, n_steps: int, delay_mode: int, delays_ptr, levels_ptr: int, depth: int) -> int:
    return lib().at_step_levels(h, n_steps, delay_mode, _vp(delays_ptr), _vp(levels_ptr), depth)


def at_set_history(h, levels_ptr: int, depth: int, level: int) -> int:
    return lib().at_set_history(h, _vp(levels_ptr), depth, level)


def at_checkpoint_bytes(h, n_steps: int, interval: int) -> int:
    return int(lib().at_checkpoint_bytes(h, n_steps, interval))


def at_step_checkpointed(h, n_steps: int, delay_mode: int, delays_ptr, interval: int, ckpt_ptr: int) -> int:
    return lib().at_step_checkpointed(h, n_steps, delay_mode, _vp(delays_ptr), interval, _vp(ckpt_ptr))


def at_adjoint_workspace_bytes(h, interval: int) -> int:
    return int(lib().at_adjoint_workspace_bytes(h, interval))


def at_adjoint(h, n_steps: int, delay_mode: int, delays_ptr, interval: int, ckpt_ptr: int, ws_ptr: int,
               ws_bytes: int, lam_ptr: int):
    """Returns (code, dJ/dnu); lam_ptr holds dJ/du(T) on entry and dJ/du0 on return."""
    dnu = ctypes.c_double()
    rc = lib().at_adjoint(h, n_steps, delay_mode, _vp(delays_ptr), interval, _vp(ckpt_ptr), _vp(ws_ptr), ws_bytes,
                          _vp(lam_ptr), ctypes.byref(dnu))
    return rc, dnu.value


def at_last_error() -> str:
    s = lib().at_last_error()
    return s.decode() if s else ""
