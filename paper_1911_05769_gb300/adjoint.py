"""Gradients through the AT time stepper: a ``torch.autograd.Function`` whose
forward is ``at_step_checkpointed`` and whose backward is ``at_adjoint`` (the
hand-written adjoint kernel with checkpointed recomputation).  Argument
marshalling only; both directions run in the CUDA library.
"""
from __future__ import annotations

import math

from . import binding as B
from .solver import Solver


def _torch():
    import torch
    return torch


class _ATRun:
    """Holder of the autograd Function (built on first use so that importing
    the package does not import torch)."""
    fn = None

    @classmethod
    def get(cls):
        if cls.fn is None:
            torch = _torch()

            class ATRun(torch.autograd.Function):
                @staticmethod
                def forward(ctx, u0, nu, cfg):
                    dtype = "f64" if u0.dtype == torch.float64 else "f32"
                    s = Solver(u0.numel(), cfg["P"], cfg["order"], cfg["L"], float(nu), cfg["dt"], dtype=dtype,
                               length=cfg["length"], origin=cfg["origin"], forcing_amp=cfg["forcing_amp"],
                               seed=cfg["seed"], flags=cfg["flags"], max_ctas=cfg["max_ctas"], stages=cfg["stages"],
                               steps_per_pass=cfg["steps_per_pass"], device=u0.device.index)
                    s.set_state(u0.detach())
                    n, interval, mode = cfg["n_steps"], cfg["interval"], cfg["mode"]
                    ckpt = torch.empty(B.at_checkpoint_bytes(s.h, n, interval), dtype=torch.uint8, device=s.device)
                    delays = cfg.get("delays")
                    if mode == B.AT_FREE:
                        delays = torch.full((n, cfg["P"], 2), -1, dtype=torch.int8, device=s.device)
                    rc = B.at_step_checkpointed(s.h, n, mode, delays.data_ptr() if delays is not None else None,
                                                interval, ckpt.data_ptr())
                    if rc != B.AT_OK:
                        raise B.AtError(rc, "at_step_checkpointed")
                    ctx.solver, ctx.ckpt, ctx.delays, ctx.cfg = s, ckpt, delays, cfg
                    ctx.nu_meta = (nu.dtype, nu.device)
                    return s.state()

                @staticmethod
                def backward(ctx, grad_uT):
                    s, cfg = ctx.solver, ctx.cfg
                    mode = B.AT_REPLAY if cfg["mode"] == B.AT_FREE else cfg["mode"]
                    lam = grad_uT.detach().to(s.tdtype).contiguous().clone()
                    nbytes = B.at_adjoint_workspace_bytes(s.h, cfg["interval"])
                    ws = torch.empty(nbytes, dtype=torch.uint8, device=s.device)
                    d = ctx.delays
                    rc, dnu = B.at_adjoint(s.h, cfg["n_steps"], mode, d.data_ptr() if d is not None else None,
                                           cfg["interval"], ctx.ckpt.data_ptr(), ws.data_ptr(), nbytes,
                                           lam.data_ptr())
                    if rc != B.AT_OK:
                        raise B.AtError(rc, "at_adjoint")
                    s.close()
                    ctx.solver = None
                    dt_, dev_ = ctx.nu_meta
                    return lam, torch.tensor(dnu, dtype=dt_, device=dev_), None

            cls.fn = ATRun
        return cls.fn


def at_run(u0, nu, *, P, order, L, dt, n_steps, mode=B.AT_SEEDED, seed=0, interval=100, delays=None,
           length=2 * math.pi, origin=0.0, forcing_amp=0.0, flags=0, max_ctas=0, stages=0, steps_per_pass=0):
    """u(n_steps) of the AT run from ``u0`` (a CUDA tensor, float32 or float64)
    with viscosity ``nu`` (a 0-d tensor); differentiable with respect to both.

    ``mode``: AT_SEEDED (delays from ``seed``), AT_SYNC, AT_REPLAY (``delays``:
    int8 CUDA tensor [n_steps, P, 2]) or AT_FREE (delays recorded on the forward
    run and replayed by the adjoint).  Checkpoints every ``interval`` levels.
    """
    cfg = dict(P=P, order=order, L=L, dt=dt, n_steps=n_steps, mode=mode, seed=seed, interval=interval,
               delays=delays, length=length, origin=origin, forcing_amp=forcing_amp, flags=flags,
               max_ctas=max_ctas, stages=stages, steps_per_pass=steps_per_pass)
    return _ATRun.get().apply(u0, nu, cfg)
