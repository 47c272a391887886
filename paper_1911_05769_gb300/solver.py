"""Convenience wrapper over the C ABI: the workspace lives in a torch tensor.

torch provides only device memory and the stream; every step of the method
runs in the CUDA library.
"""
from __future__ import annotations

import math

from . import binding as B


class Solver:
    """One 1D problem: N points, P subdomains, order 2|4, maximal delay L.

    ``dtype`` is "f64" or "f32".  ``stream`` defaults to torch's current
    stream on the current device.
    """

    def __init__(self, N, P, order, L, nu, dt, *, dtype="f64", length=2 * math.pi, origin=0.0,
                 forcing_amp=0.0, seed=0, flags=0, timeout_ns=0, max_ctas=0, stages=0,
                 test_skip_step=0, steps_per_pass=0, stream=None, device=None):
        import torch
        self.torch = torch
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        g = B.at_grid()
        g.dim, g.bc = 1, B.AT_BC_PERIODIC
        g.dtype = B.AT_F64 if dtype == "f64" else B.AT_F32
        g.flags = flags
        g.n[0], g.n[1], g.n[2] = N, 1, 1
        g.length[0] = length
        g.origin[0] = origin
        g.forcing_amp = forcing_amp
        g.seed = seed & (2 ** 64 - 1)
        g.timeout_ns = timeout_ns
        g.max_ctas = max_ctas
        g.stages = stages
        g.test_skip_step = test_skip_step
        g.steps_per_pass = steps_per_pass
        nbytes = B.at_workspace_bytes(g, P, order, L)
        if nbytes == 0:
            raise B.AtError(B.AT_ERR_ARG, "at_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        g.workspace = self.workspace.data_ptr()
        g.workspace_bytes = nbytes
        g.stream = self.stream.cuda_stream
        self.grid = g
        rc, h = B.at_create(g, P, order, L, nu, dt)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_create")
        self.h = h
        self.N, self.P, self.order, self.L = N, P, order, L
        self.faces = 2

    def tune(self, n_steps, mode=B.AT_FREE):
        """Runs the launch-shape autotuner (at_tune) and returns its result.
        The state advances while shapes are timed: set it again afterwards."""
        rc, res = B.at_tune(self.h, n_steps, mode)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_tune")
        return res

    def info(self):
        rc, info = B.at_get_info(self.h)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_get_info")
        return info

    def set_state(self, u):
        """u: torch tensor (device or host) or numpy array of N words."""
        t = self._as_tensor(u)
        rc = B.at_set_state(self.h, t.data_ptr())
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_set_state")
        self._keep = t     # keep a host source alive until the stream passes the copy

    def step(self, n_steps, mode=B.AT_SEEDED, delays=None):
        """delays: int8 device tensor [n_steps, P, faces] (input for REPLAY, record otherwise)."""
        ptr = None
        if delays is not None:
            assert delays.dtype == self.torch.int8 and delays.is_cuda and delays.is_contiguous()
            assert delays.numel() == n_steps * self.P * self.faces
            ptr = delays.data_ptr()
        rc = B.at_step(self.h, n_steps, mode, ptr)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_step")

    def state(self, out=None):
        """Copies the state into ``out`` (new device tensor by default); raises on a device timeout."""
        if out is None:
            out = self.torch.empty(self.N, dtype=self.tdtype, device=self.device)
        rc = B.at_state(self.h, out.data_ptr())
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_state")
        return out

    def state_error(self, out=None):
        """Compensated state only: the lo words (rounding errors of ``state()``),
        so that state() + state_error() is the value carried."""
        if out is None:
            out = self.torch.empty(self.N, dtype=self.tdtype, device=self.device)
        rc = B.at_state_error(self.h, out.data_ptr())
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_state_error")
        return out

    def status(self):
        return B.at_status(self.h)

    def delay_stats(self):
        rc, hist, m1, m2 = B.at_delay_stats(self.h, self.L)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_delay_stats")
        return hist, m1, m2

    def close(self):
        if getattr(self, "h", None) is not None:
            B.at_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _as_tensor(self, u):
        torch = self.torch
        if not isinstance(u, torch.Tensor):
            u = torch.from_numpy(u)
        if u.dtype != self.tdtype:
            u = u.to(self.tdtype)
        u = u.contiguous()
        if u.numel() != self.N:
            raise ValueError(f"state needs {self.N} values, got {u.numel()}")
        return u


class EnsembleSolver(Solver):
    """Many independent 1D problems of M-point subdomains in one persistent launch.

    ``instances`` is a sequence of dicts with keys n, L, nu, dt and optionally
    bc (default AT_BC_EXACT_TANH), length (2 pi), origin (-pi), tanh_a,
    tanh_c, tanh_xc, seed.  The state is the concatenation of the instances'
    fields; step/state/delay_stats work as for ``Solver`` over all P = N / M
    subdomains.
    """

    def __init__(self, instances, M, order, *, dtype="f32", flags=0, timeout_ns=0, max_ctas=0, stages=0,
                 steps_per_pass=0, tile_subdomains=0, stream=None, device=None):
        import torch
        self.torch = torch
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        arr = (B.at_instance * len(instances))()
        for a, d in zip(arr, instances):
            a.n, a.L = int(d["n"]), int(d["L"])
            a.bc = int(d.get("bc", B.AT_BC_EXACT_TANH))
            a.length = float(d.get("length", 2 * math.pi))
            a.origin = float(d.get("origin", -math.pi))
            a.nu, a.dt = float(d["nu"]), float(d["dt"])
            a.tanh_a = float(d.get("tanh_a", 0.0))
            a.tanh_c = float(d.get("tanh_c", 0.0))
            a.tanh_xc = float(d.get("tanh_xc", 0.0))
            a.seed = int(d.get("seed", 0)) & (2 ** 64 - 1)
        g = B.at_grid()
        g.dim = 1
        g.dtype = B.AT_F64 if dtype == "f64" else B.AT_F32
        g.flags = flags
        g.timeout_ns = timeout_ns
        g.max_ctas = max_ctas
        g.stages = stages
        g.steps_per_pass = steps_per_pass
        g.tile_subdomains = tile_subdomains
        nbytes = B.at_batch_workspace_bytes(g, arr, M, order)
        if nbytes == 0:
            raise B.AtError(B.AT_ERR_ARG, "at_batch_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        g.workspace = self.workspace.data_ptr()
        g.workspace_bytes = nbytes
        g.stream = self.stream.cuda_stream
        self.grid = g
        self.instances = arr
        rc, h = B.at_create_batch(g, arr, M, order)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_create_batch")
        self.h = h
        self.faces = 2
        self.N = sum(int(d["n"]) for d in instances)
        self.P = self.N // M
        self.order = order
        self.L = max(int(d["L"]) for d in instances)
        self.offsets = [0]
        for d in instances:
            self.offsets.append(self.offsets[-1] + int(d["n"]))


class Solver3D(Solver):
    """Scalar 3D Burgers on a periodic box of n = (n0, n1, n2) points (x fastest)
    in subdomains of sub = (m0, m1, m2) points, order 2, six AT faces per
    subdomain.  The state is a flat tensor of n0 n1 n2 words (or shaped
    (n2, n1, n0)); delays are [n_steps, P, 6].  steps_per_pass > 1: AT_FREE
    steps advance each subdomain that many levels per pass (at most L + 1)."""

    def __init__(self, n, sub, L, nu, dt, *, dtype="f32", length=(2 * math.pi,) * 3, seed=0, flags=0,
                 timeout_ns=0, max_ctas=0, stages=0, steps_per_pass=0, test_skip_step=0, stream=None, device=None):
        import torch
        self.torch = torch
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        g = B.at_grid()
        g.dim, g.bc = 3, B.AT_BC_PERIODIC
        g.dtype = B.AT_F64 if dtype == "f64" else B.AT_F32
        g.flags = flags
        for a in range(3):
            g.n[a] = int(n[a])
            g.sub[a] = int(sub[a])
            g.length[a] = float(length[a])
        g.seed = seed & (2 ** 64 - 1)
        g.timeout_ns = timeout_ns
        g.max_ctas = max_ctas
        g.stages = stages
        g.steps_per_pass = steps_per_pass
        g.test_skip_step = test_skip_step
        P = 1
        for a in range(3):
            P *= int(n[a]) // int(sub[a])
        nbytes = B.at_workspace_bytes(g, P, 2, L)
        if nbytes == 0:
            raise B.AtError(B.AT_ERR_ARG, "at_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        g.workspace = self.workspace.data_ptr()
        g.workspace_bytes = nbytes
        g.stream = self.stream.cuda_stream
        self.grid = g
        rc, h = B.at_create(g, P, 2, L, nu, dt)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_create")
        self.h = h
        self.N = int(n[0]) * int(n[1]) * int(n[2])
        self.P, self.order, self.L = P, 2, L
        self.faces = 6
        self.shape = (int(n[2]), int(n[1]), int(n[0]))


class System3D(Solver3D):
    """The 3D system of Eq. BS: velocity (u, v, w) and 0..2 passive scalars,
    ``kappa`` = (nu, nu, nu, alpha_1, ...).  The state holds the fields one
    after another (shape (nfields, n2, n1, n0)); delays are [n_steps, P, 6]."""

    def __init__(self, n, sub, L, kappa, dt, *, dtype="f32", length=(2 * math.pi,) * 3, seed=0, flags=0,
                 timeout_ns=0, max_ctas=0, stages=0, stream=None, device=None):
        import torch
        self.torch = torch
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        g = B.at_grid()
        g.dim, g.bc = 3, B.AT_BC_PERIODIC
        g.dtype = B.AT_F64 if dtype == "f64" else B.AT_F32
        g.flags = flags
        for a in range(3):
            g.n[a] = int(n[a])
            g.sub[a] = int(sub[a])
            g.length[a] = float(length[a])
        g.seed = seed & (2 ** 64 - 1)
        g.timeout_ns = timeout_ns
        g.max_ctas = max_ctas
        g.stages = stages
        P = 1
        for a in range(3):
            P *= int(n[a]) // int(sub[a])
        nf = len(kappa)
        nbytes = B.at_system_workspace_bytes(g, P, L, nf)
        if nbytes == 0:
            raise B.AtError(B.AT_ERR_ARG, "at_system_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        g.workspace = self.workspace.data_ptr()
        g.workspace_bytes = nbytes
        g.stream = self.stream.cuda_stream
        self.grid = g
        rc, h = B.at_create_system(g, P, L, list(kappa), dt)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_create_system")
        self.h = h
        self.nfields = nf
        self.N = nf * int(n[0]) * int(n[1]) * int(n[2])
        self.P, self.order, self.L = P, 2, L
        self.faces = 6
        self.shape = (nf, int(n[2]), int(n[1]), int(n[0]))

    def moments(self):
        """[(mean, mean square)] per field (FP64 sums on the device)."""
        rc, m = B.at_moments(self.h, self.nfields)
        if rc != B.AT_OK:
            raise B.AtError(rc, "at_moments")
        return m
