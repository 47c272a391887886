#!/usr/bin/env python3
"""Benchmark: grid-point updates per second of the weakly-synchronous AT
solver on the forced 1D Burgers workload N = 2^26 points, P = 65536
subdomains of 1024, 4th-order stencils, L = 3, FP32 state (arXiv 1911.05769
method; synthetic seeded initial field, 64 Fourier modes with k^-1 amplitudes).

A bench step is one at_step call that advances the whole field by
--time-steps time steps (default 1000) in one persistent kernel launch.  The
headline arm runs free-running delays (Algorithm 2: a CTA waits only when a
neighbour lags by more than L); the synchronous arm (grid barrier every step,
Algorithm 1) and the seeded-delay arm are timed in the same process.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import at_workloads as W  # noqa: E402

WORKLOAD = "burgers1d_forced_n2p26"
METRIC = "grid-point updates/sec (GPts/s), AT vs synchronous, 1D forced Burgers N=2^26 order 4 L=3"
UNIT = "GPts/s"
FALLBACK_HBM = 6800.0
KERNEL_SOURCES = ["paper_1911_05769_gb300/csrc/at_kernels.cuh", "paper_1911_05769_gb300/csrc/at_device.cuh",
                  "paper_1911_05769_gb300/csrc/at_kernels_f32.cu"]
PROFILE = os.path.join(ROOT, "profiles", "at_stepper_f32_o4_n2p26.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--time-steps", type=int, default=1000, help="time steps per bench step (one launch)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-extra", action="store_true", help="skip the f64, e2e and CPU-baseline legs")
    ap.add_argument("--cpu-sample-steps", type=int, default=100)
    ap.add_argument("--cpu-sample-subdomains", type=int, default=4096)
    ap.add_argument("--ctas", type=int, default=0, help="CTAs of the persistent kernel (0 = one per SM)")
    ap.add_argument("--stages", type=int, default=0, help="tiles in flight per CTA (0 = default)")
    ap.add_argument("--arms", default="all",
                    help="timed arms besides the headline free_blocked: all or a comma list of "
                         "sync,sync_blocked,seeded,free")
    ap.add_argument("--N", type=int, default=0, help="smaller N for profiling runs (P scales, M stays 1024)")
    ap.add_argument("--spp", type=int, default=-1,
                    help="levels per pass of the free-running arm (temporal blocking); -1 = L+1")
    ap.add_argument("--M", type=int, default=0, help="points per subdomain for experiments (default 1024)")
    ap.add_argument("--order", type=int, default=0, help="stencil order for experiments (default 4)")
    ap.add_argument("--forcing", type=float, default=-1.0, help="forcing amplitude for experiments (default 0.1)")
    ap.add_argument("--ensemble-only", action="store_true", help="time only the 2048-instance ensemble leg")
    ap.add_argument("--ens-time-steps", type=int, default=5000, help="time steps per ensemble launch")
    ap.add_argument("--no-tune", action="store_true", help="ensemble leg: keep the default launch shape")
    ap.add_argument("--ens-shape", default="",
                    help="ensemble leg without tuning, shape K,spp,stages,ctas (subdomains per tile, levels per "
                         "pass of the free arm, tile buffers, CTAs), for profiling runs")
    ap.add_argument("--adjoint-only", action="store_true", help="time only the adjoint leg")
    ap.add_argument("--only-3d", action="store_true", help="time only the 3D leg")
    ap.add_argument("--only-system", action="store_true", help="time only the 3D system leg")
    ap.add_argument("--time-steps-3d", type=int, default=500, help="time steps per 3D launch")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def sources_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """Per-launch DRAM bytes of the stepper from the committed ncu summary,
    or None if absent or taken on other kernel sources."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None, None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"kernel_sources_sha:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != sources_sha():
        return None, None
    t = re.search(r"time_steps_per_launch:\s*([0-9]+)", txt)
    return float(m.group(1)), int(t.group(1)) if t else None


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        loaded = [x for x in sm if smax and x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def max_over_ranks(pg, x: float, device) -> float:
    """The largest x over the ranks of process group module `pg` (None: one
    process); the job's time is its slowest rank's."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput in G units/s: every rank processes the same units
    (weak scaling), the job takes the slowest rank's time."""
    return ws * units_per_rank / seconds / 1e9


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gpu" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return ws, rank, local, pg


def compiler_version() -> str:
    try:
        return subprocess.check_output(["gcc", "--version"], text=True).splitlines()[0]
    except Exception:
        return "gcc (version unknown)"


def cpu_baseline(args, u0, dt, cfg):
    """The oracle as it stands, timed on the host cores: single-threaded on a
    window of 512 subdomains and with OpenMP over subdomains on every core on
    a window of 4096 subdomains, both over 100 seeded steps of the workload,
    median of 5 repetitions (after one untimed run)."""
    import oracle
    oracle.build()
    N, P, M = cfg["N"], cfg["P"], cfg["N"] // cfg["P"]
    steps = args.cpu_sample_steps
    ncores = os.cpu_count() or 1

    def timed(nsub, threads, reps=5):
        oracle.threads(threads)
        u0w = np.ascontiguousarray(u0[:nsub * M], dtype=np.float64)
        kw = dict(N=N, P=P, order=cfg["order"], L=cfg["L"], nu=cfg["nu"], dt=dt, n_steps=steps,
                  forcing_amp=cfg["forcing_amp"], delay_mode=oracle.SEEDED, seed=cfg["seed"], p_lo=0, p_count=nsub)
        oracle.run(u0w, **kw)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle.run(u0w, **kw)
            ts.append(time.perf_counter() - t0)
        med = statistics.median(ts)
        return nsub * M * steps / med / 1e9, med, ts

    one, one_s, _ = timed(min(512, P), 1)
    nsub = min(args.cpu_sample_subdomains, P)
    used = oracle.threads(ncores)
    allc, all_s, _ = timed(nsub, used)
    out = {"value": allc, "unit": UNIT, "cores": used, "kind": "oracle",
           "sample": f"{nsub} subdomains x {M} points of the N=2^26 workload, {steps} seeded-delay steps, FP64, "
                     f"OpenMP over subdomains on {used} threads (nproc {ncores}): median of 5 runs {all_s:.3f} s",
           "nproc": ncores, "compiler": compiler_version(), "repetitions": 5,
           "single_thread": {"value": one, "unit": UNIT, "cores": 1,
                             "sample": f"{min(512, P)} subdomains x {M} points, {steps} seeded steps: "
                                       f"median of 5 runs {one_s:.3f} s"}}
    return out


def window_oracles(args, u0, dt, cfg, recs):
    """FP64 oracle runs of a window of the workload's subdomains (all host
    cores): synchronous, seeded, every delay at L (the c15 envelope's
    reference), and the recorded delays of each free-running arm replayed."""
    import oracle
    oracle.build()
    oracle.threads(os.cpu_count() or 1)
    N, P, M = cfg["N"], cfg["P"], cfg["N"] // cfg["P"]
    nsub = min(args.cpu_sample_subdomains, P)
    steps = args.cpu_sample_steps
    u0w = np.ascontiguousarray(u0[:nsub * M], dtype=np.float64)
    kw = dict(N=N, P=P, order=cfg["order"], L=cfg["L"], nu=cfg["nu"], dt=dt, n_steps=steps,
              forcing_amp=cfg["forcing_amp"], p_lo=0, p_count=nsub)
    out = {"sync": oracle.run(u0w, delay_mode=oracle.SYNC, **kw)[0],
           "seeded": oracle.run(u0w, delay_mode=oracle.SEEDED, seed=cfg["seed"], **kw)[0],
           "k_eq_L": oracle.run(u0w, delay_mode=oracle.REPLAY,
                                replay=np.full((steps, nsub, 2), cfg["L"], np.int8), **kw)[0]}
    for name, rec in recs.items():
        out[name] = oracle.run(u0w, delay_mode=oracle.REPLAY, replay=np.ascontiguousarray(rec[:, :nsub, :]), **kw)[0]
    return out, nsub, steps


def small_config(args, at, torch, dev, stream):
    """N = 4096, P = 16, order 2, L = 2, nu = 0.02, FP64, u0 = sin x + 0.5 sin(3x+1):
    1000-step launches, free-running (plain and in passes of L+1 levels) vs
    seeded vs synchronous, microseconds per step."""
    cfg = W.config("burgers1d_n4096")
    u0 = W.initial_field(cfg)
    _, dx = W.grid(cfg["N"])
    dt = W.dt_rule(u0, dx, cfg["nu"])
    u0_dev = torch.from_numpy(u0).to(dev)
    res = {"workload": "burgers1d_n4096", "N": cfg["N"], "P": cfg["P"], "order": cfg["order"], "L": cfg["L"],
           "dtype": "f64", "time_steps_per_launch": cfg["n_steps"]}
    arms = (("free", at.AT_FREE, 0), ("free_blocked", at.AT_FREE, cfg["L"] + 1), ("seeded", at.AT_SEEDED, 0),
            ("sync", at.AT_SYNC, 0), ("sync_blocked", at.AT_SYNC, cfg["L"] + 1))
    for name, mode, spp in arms:
        s = at.Solver(cfg["N"], cfg["P"], cfg["order"], cfg["L"], cfg["nu"], dt, dtype="f64", seed=cfg["seed"],
                      stream=stream, device=dev.index, steps_per_pass=spp)
        s.set_state(u0_dev)
        for _ in range(2):
            s.step(cfg["n_steps"], mode)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                s.step(cfg["n_steps"], mode)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        us_step = 1e3 * ms / (reps * cfg["n_steps"])
        res[name] = {"us_per_step": us_step, "value": cfg["N"] / (us_step * 1e-6) / 1e9, "unit": UNIT}
        s.close()
    res["speedup_free_over_sync"] = res["sync"]["us_per_step"] / res["free"]["us_per_step"]
    res["speedup_free_blocked_over_sync_blocked"] = res["sync_blocked"]["us_per_step"] / res["free_blocked"]["us_per_step"]
    return res


def ensemble_config(args, at, torch, dev, stream):
    """The 2048-instance travelling-wave ensemble (N_j log-uniform in
    [2^10, 2^16], M = 256, order 2, L_j in {1, 2, 3}, FP32): one persistent
    launch of 5000 steps captured in a CUDA graph and replayed, launch shape
    picked by the autotuner (free-running delays); the synchronous arm the same
    way; the FP32 result's error against the FP64 oracle on sampled instances."""
    inst = W.ensemble()
    M, order = 256, 2
    time_steps = args.ens_time_steps
    Ntot = sum(d["n"] for d in inst)
    u0 = torch.from_numpy(W.ensemble_field(inst)).to(device=dev, dtype=torch.float32)
    res = {"workload": "burgers1d_ensemble_2048", "instances": len(inst), "N": Ntot, "P": Ntot // M, "M": M,
           "order": order, "L_j": [1, 2, 3], "dtype": "f32", "time_steps_per_launch": time_steps,
           "l2": f"state {Ntot * 4 / 2**20:.0f} MiB: close to the 126 MiB L2 (replays continue in place)"}
    Lmax = max(d["L"] for d in inst)

    shape = [int(x) for x in args.ens_shape.split(",")] if args.ens_shape else None

    def run(mode, name, spp=None, flags=0):
        kw = {}
        if shape:
            # (the compensated kernels hold fewer CTAs per SM: all that fit)
            kw = dict(tile_subdomains=shape[0], stages=shape[2],
                      max_ctas=0 if flags & at.AT_FLAG_COMPENSATED else shape[3])
            if mode == at.AT_FREE and spp is None:
                spp = shape[1]
        s = at.EnsembleSolver(inst, M, order, dtype="f32", stream=stream, device=dev.index, flags=flags,
                              steps_per_pass=(Lmax + 1 if mode == at.AT_FREE else 0) if spp is None else spp, **kw)
        with torch.cuda.stream(stream):
            s.set_state(u0)
        t = None if (args.no_tune or shape) else s.tune(200, mode)
        with torch.cuda.stream(stream):
            s.set_state(u0)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            s.step(time_steps, mode)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g.replay()
            ev[0].record(stream)
            for _ in range(args.steps):
                g.replay()
            ev[1].record(stream)
        torch.cuda.synchronize(dev)
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        rc = s.status()
        if rc != at.AT_OK:
            raise RuntimeError(f"ensemble {name}: device status {rc}: {at.at_last_error()}")
        info = s.info()
        assert info.step == (args.warmup + args.steps) * time_steps, info.step
        s.close()
        del g
        return {"value": Ntot * time_steps / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_launch": ms,
                "shape": {"ctas": info.ctas, "stages": info.stages, "steps_per_pass": info.steps_per_pass,
                          "tile_subdomains": info.tile_subdomains},
                "tuned": None if t is None else {
                    "shapes_tried": t.n_tried, "ms_200_steps_first": t.first_ms, "ms_200_steps_best": t.best_ms}}

    res["free"] = run(at.AT_FREE, "free")
    res["sync"] = run(at.AT_SYNC, "sync")
    res["sync_blocked"] = run(at.AT_SYNC, "sync_blocked", spp=Lmax + 1)
    res["free_compensated"] = run(at.AT_FREE, "free_compensated", flags=at.AT_FLAG_COMPENSATED)
    res["speedup_free_over_sync"] = res["free"]["value"] / res["sync"]["value"]
    res["speedup_free_over_sync_blocked"] = res["free"]["value"] / res["sync_blocked"]["value"]
    res["effective_one_pass_frac"] = res["free"]["value"] * 1e9 * 8 / (hbm_peak()[0] * 1e9)
    # algorithmic bytes per update with passes of the launch's steps_per_pass
    # (warps whose smallest L_j is lower take shorter passes and move more:
    # this is the least the free-running arm can move)
    spp = max(1, res["free"]["shape"]["steps_per_pass"])
    w, R, s_lev = 4, order // 2, order // 2 + 1
    bpu = (2 * w + 2 * R * s_lev * w / M) / spp + 2 * R * w / M
    peak, src = hbm_peak()
    res["roofline"] = {"bound": "hbm", "algorithmic_bytes_per_update": bpu,
                       "achieved": res["free"]["value"] * bpu, "peak": peak, "unit": "GB/s",
                       "frac": res["free"]["value"] * bpu / peak, "peak_source": src,
                       "note": "bound by per-tile latency and control instructions, not by HBM"}
    res["gpu_launches_per_replay"] = 1
    # FP32 error against the FP64 oracle after the full 5000 seeded steps, on
    # the four smallest instances (the largest dt), one mid-size one and the
    # largest: plain FP32 state and the compensated state (hi + lo)
    n = np.array([d["n"] for d in inst])
    which = list(np.argsort(n)[:4]) + [int(np.argsort(n)[len(n) // 2]), int(np.argmax(n))]
    finals = {}
    for key, fl in (("plain", 0), ("compensated", at.AT_FLAG_COMPENSATED)):
        s = at.EnsembleSolver(inst, M, order, dtype="f32", stream=stream, device=dev.index, flags=fl)
        with torch.cuda.stream(stream):
            s.set_state(u0)
            s.step(time_steps, at.AT_SEEDED)
            g = s.state().double().cpu().numpy()
            if fl:
                g = g + s.state_error().double().cpu().numpy()
        s.close()
        finals[key] = g
    import oracle
    oracle.build()
    oracle.threads(os.cpu_count() or 1)
    offs = np.concatenate([[0], np.cumsum(n)])
    worst = {"plain": 0.0, "compensated": 0.0}
    for j in which:
        d = inst[j]
        ref, _ = oracle.run(W.instance_field(d), N=d["n"], P=d["n"] // M, order=order, L=d["L"], nu=d["nu"],
                            dt=d["dt"], n_steps=time_steps, x0=d["origin"], dx=d["length"] / d["n"],
                            bc=oracle.BC_TANH, tanh=(d["tanh_a"], d["tanh_c"], d["tanh_xc"]),
                            delay_mode=oracle.SEEDED, seed=d["seed"])
        for key, g in finals.items():
            part = g[offs[j]:offs[j + 1]]
            worst[key] = max(worst[key], float(np.max(np.abs(part - ref)) / np.max(np.abs(ref))))
    res["err_vs_fp64_oracle"] = {"rel_linf": worst["compensated"], "state": "compensated (hi + lo)",
                                 "rel_linf_plain_fp32": worst["plain"], "mode": "seeded", "steps": time_steps,
                                 "instances": [int(j) for j in which]}
    return res


def adjoint_config(args, at, torch, dev):
    """Gradient of ||u(T) - u_target||^2 with respect to u0 (2^20 values) and
    nu through 2000 seeded AT steps (order 2, L = 2, nu = 0.01, checkpoints
    every 100): forward (checkpointed) and backward (recomputation + adjoint
    kernel) timed with CUDA events; the FP64 gradient checked against central
    differences of the FP64 forward run on 16 random directions."""
    wl = W.adjoint_workload()
    N, n_steps = wl["N"], wl["n_steps"]
    stream = torch.cuda.current_stream(dev)

    def forward_run(u0, nu, dtype="f64"):
        s = at.Solver(N, wl["P"], wl["order"], wl["L"], nu, wl["dt"], dtype=dtype, seed=wl["seed"], device=dev.index)
        s.set_state(torch.as_tensor(u0).to(dev))
        s.step(n_steps, at.AT_SEEDED)
        out = s.state().double()
        s.close()
        return out

    target = forward_run(wl["u0_target"], wl["nu_target"])
    res = {"workload": wl["name"], "N": N, "P": wl["P"], "order": wl["order"], "L": wl["L"], "nu": wl["nu"],
           "time_steps": n_steps, "checkpoint_interval": wl["interval"], "loss": "||u(T) - u_target||^2"}

    def grad(dtype, reps):
        tdt = torch.float64 if dtype == "f64" else torch.float32
        u0 = torch.from_numpy(wl["u0"]).to(device=dev, dtype=tdt).requires_grad_(True)
        nu = torch.tensor(wl["nu"], dtype=torch.float64, device=dev, requires_grad=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fwd, bwd = [], []
        for r in range(reps + 1):
            ev[0].record(stream)
            uT = at.at_run(u0, nu, P=wl["P"], order=wl["order"], L=wl["L"], dt=wl["dt"], n_steps=n_steps,
                           mode=at.AT_SEEDED, seed=wl["seed"], interval=wl["interval"])
            ev[1].record(stream)
            loss = ((uT.double() - target) ** 2).sum()
            gu0, gnu = torch.autograd.grad(loss, (u0, nu))
            ev[2].record(stream)
            torch.cuda.synchronize(dev)
            if r > 0:
                fwd.append(ev[0].elapsed_time(ev[1]))
                bwd.append(ev[1].elapsed_time(ev[2]))
        f, b = statistics.median(fwd), statistics.median(bwd)
        return gu0.double(), float(gnu), {"forward_ms": f, "backward_ms": b,
                                           "value": N * n_steps / ((f + b) * 1e-3) / 1e9, "unit": UNIT,
                                           "value_note": "forward-equivalent updates per second of one gradient"}

    g32, n32, t32 = grad("f32", 3)
    g64, n64, t64 = grad("f64", 1)
    res["f32"] = t32
    res["f64"] = t64
    res["f32_vs_f64_gradient_rel_l2"] = float((g32 - g64).norm() / g64.norm())
    res["f32_vs_f64_dnu_rel"] = abs(n32 - n64) / abs(n64)
    # central differences of the FP64 forward run
    rng = np.random.default_rng(16)
    base = torch.from_numpy(wl["u0"]).to(dev)

    def J(u, n):
        return float(((forward_run(u, n) - target) ** 2).sum())

    worst = 0.0
    for _ in range(16):
        d = torch.from_numpy(rng.standard_normal(N)).to(dev)
        eps = 1e-4
        fd = (J(base + eps * d, wl["nu"]) - J(base - eps * d, wl["nu"])) / (2 * eps)
        worst = max(worst, abs(fd - float((g64 * d).sum())) / abs(fd))
    enu = 1e-2 * wl["nu"]
    fdnu = (J(base, wl["nu"] + enu) - J(base, wl["nu"] - enu)) / (2 * enu)
    res["fd_check_fp64"] = {"directions": 16, "max_rel_err_u0": worst, "rel_err_nu": abs(fdnu - n64) / abs(fdnu),
                            "dJ_dnu": n64}
    s = at.Solver(N, wl["P"], wl["order"], wl["L"], wl["nu"], wl["dt"], dtype="f32", seed=wl["seed"], device=dev.index)
    res["memory_bytes"] = {"checkpoints_f32": at.at_checkpoint_bytes(s.h, n_steps, wl["interval"]),
                           "adjoint_workspace_f32": at.at_adjoint_workspace_bytes(s.h, wl["interval"])}
    s.close()
    return res


def config3d(args, at, torch, dev):
    """3D scalar Burgers, 512^3 FP32 in 32^3 subdomains (4096), order 2, L = 2,
    nu = 5e-3, k^-5/3 field (seed 4): launches of 500 steps (4 per 2000-step
    run), free-running in passes of L + 1 levels vs free-running one level per
    pass vs seeded vs synchronous; the FP32 error against the FP64 oracle over
    all 2000 steps on a 128^3 box at the workload's dx, nu and dt (seeded, and
    free-running in passes of L + 1 levels with its recorded delays)."""
    n, sub, L, nu = 512, (32, 32, 32), 2, 5e-3
    u0 = W.u0_spectral3d(n, seed=4, kmax=32)
    dt = W.dt_rule(u0, 2 * np.pi / n, nu, dim=3)
    u0_dev = torch.from_numpy(u0.ravel()).to(device=dev, dtype=torch.float32)
    del u0
    S = args.time_steps_3d
    N = n ** 3
    res = {"workload": "burgers3d_n512", "n": n, "sub": list(sub), "P": (n // sub[0]) ** 3, "L": L, "nu": nu,
           "dt": dt, "dtype": "f32", "time_steps_per_launch": S}
    stream = torch.cuda.Stream(device=dev)
    for name, mode, spp in (("free", at.AT_FREE, L + 1), ("free_one_level_per_pass", at.AT_FREE, 1),
                            ("seeded", at.AT_SEEDED, 1), ("sync", at.AT_SYNC, 1)):
        s = at.Solver3D((n, n, n), sub, L, nu, dt, dtype="f32", seed=5, stream=stream, device=dev.index,
                        steps_per_pass=spp)
        with torch.cuda.stream(stream):
            s.set_state(u0_dev)
            s.step(S, mode)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = max(1, min(args.steps, 4))
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for _ in range(reps):
                s.step(S, mode)
            ev[1].record(stream)
        torch.cuda.synchronize(dev)
        ms = ev[0].elapsed_time(ev[1]) / reps
        rc = s.status()
        if rc != at.AT_OK:
            raise RuntimeError(f"3D {name}: device status {rc}: {at.at_last_error()}")
        fin = s.state()
        info = s.info()
        hist, m1, _ = s.delay_stats()
        res[name] = {"value": N * S / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_launch": ms, "mean_k": m1,
                     "max_abs_u": float(fin.abs().max()), "ctas": info.ctas, "threads": info.threads,
                     "levels_per_pass": spp}
        s.close()
    res["speedup_free_over_sync"] = res["free"]["value"] / res["sync"]["value"]
    res["speedup_free_one_level_per_pass_over_sync"] = res["free_one_level_per_pass"]["value"] / res["sync"]["value"]
    # algorithmic bytes per update: state read + write once per pass of b
    # levels; per pass each subdomain writes its 6 faces at 2 levels (the
    # last two of the pass) and reads 2 levels of its neighbours' 6 faces
    # (one level per pass: 6 faces written, 2 levels of 6 read)
    b = L + 1
    bpu = (2 * 4 + 24 * 4 / sub[0]) / b
    bpu1 = 2 * 4 + 18 * 4 / sub[0]
    peak, src = hbm_peak()
    res["roofline"] = {"bound": "hbm", "algorithmic_bytes_per_update": bpu,
                       "achieved": res["free"]["value"] * bpu, "peak": peak, "unit": "GB/s",
                       "frac": res["free"]["value"] * bpu / peak, "peak_source": src,
                       "one_level_per_pass": {"algorithmic_bytes_per_update": bpu1,
                                              "frac": res["free_one_level_per_pass"]["value"] * bpu1 / peak}}
    # FP32 against the FP64 oracle over all 2000 steps at the workload's dx,
    # nu and dt: a periodic 128^3 box of length pi/2 (32^3 subdomains, the
    # k^-5/3 recipe at the workload's wavenumbers), seeded delays
    import oracle
    oracle.build()
    oracle.threads(os.cpu_count() or 1)
    nb, box, nsteps = 128, np.pi / 2, 2000
    ub = W.u0_spectral3d(nb, seed=4, kmax=8)
    dtb = W.dt_rule(ub, box / nb, nu, dim=3)
    s = at.Solver3D((nb, nb, nb), sub, L, nu, dtb, dtype="f32", seed=5, device=dev.index, length=(box,) * 3)
    s.set_state(torch.from_numpy(ub.ravel()).to(dev))
    s.step(nsteps, at.AT_SEEDED)
    g = s.state().double().cpu().numpy().reshape(ub.shape)
    s.close()
    ref, _ = oracle.run3d(ub, P=(4, 4, 4), L=L, nu=nu, dt=dtb, n_steps=nsteps, length=box, delay_mode=oracle.SEEDED,
                          seed=5)
    res["err_vs_fp64_oracle"] = {"rel_linf": float(np.max(np.abs(g - ref)) / np.max(np.abs(ref))),
                                 "box": [nb, nb, nb], "box_length": box, "nu": nu, "dt": dtb, "steps": nsteps,
                                 "mode": "seeded"}
    # the free-running arm (passes of L + 1 levels): its recorded delays
    # replayed by the oracle
    s = at.Solver3D((nb, nb, nb), sub, L, nu, dtb, dtype="f32", seed=5, device=dev.index, length=(box,) * 3,
                    steps_per_pass=L + 1)
    s.set_state(torch.from_numpy(ub.ravel()).to(dev))
    rec = torch.full((nsteps, s.P, 6), -1, dtype=torch.int8, device=dev)
    s.step(nsteps, at.AT_FREE, rec)
    g = s.state().double().cpu().numpy().reshape(ub.shape)
    s.close()
    rec = rec.cpu().numpy()
    ref, _ = oracle.run3d(ub, P=(4, 4, 4), L=L, nu=nu, dt=dtb, n_steps=nsteps, length=box, delay_mode=oracle.REPLAY,
                          replay=rec)
    res["err_vs_fp64_oracle_free"] = {"rel_linf": float(np.max(np.abs(g - ref)) / np.max(np.abs(ref))),
                                      "steps": nsteps, "mode": "free-running, passes of L + 1 levels, replayed",
                                      "mean_k": float(rec.mean())}
    return res


def config_system(args, at, torch, dev):
    """The 3D system of Eq. BS: velocity (u, v, w) and two passive scalars on
    256^3 points in 16^3 subdomains (4096), order 2, L = 2, nu = 0.02,
    alpha = (0.01, 0.05), FP32, k^-5/3 fields (seeds 4..8) at half amplitude:
    200-step launches free-running vs seeded vs synchronous; the fields' first
    and second moments before and after; FP32 against the FP64 oracle on a
    64^3 box after 30 seeded steps."""
    n, sub, L, nf = 256, (16, 16, 16), 2, 5
    kappa = [0.02, 0.02, 0.02, 0.01, 0.05]
    q0 = np.stack([0.5 * W.u0_spectral3d(n, seed=4 + f, kmax=32) for f in range(nf)])
    dt = W.dt_rule(q0[:3].reshape(-1), 2 * np.pi / n, max(kappa), dim=3)
    q_dev = torch.from_numpy(q0.ravel()).to(device=dev, dtype=torch.float32)
    del q0
    S = 200
    npts = n ** 3
    res = {"workload": "system3d_n256_5fields", "n": n, "sub": list(sub), "P": (n // sub[0]) ** 3, "fields": nf,
           "kappa": kappa, "L": L, "dt": dt, "dtype": "f32", "time_steps_per_launch": S,
           "unit_note": "GPts/s counts grid points (all fields of a point advanced once = one update)"}
    stream = torch.cuda.Stream(device=dev)
    for name, mode in (("free", at.AT_FREE), ("seeded", at.AT_SEEDED), ("sync", at.AT_SYNC)):
        s = at.System3D((n, n, n), sub, L, kappa, dt, dtype="f32", seed=5, stream=stream, device=dev.index)
        with torch.cuda.stream(stream):
            s.set_state(q_dev)
        if name == "free":
            res["moments_initial"] = s.moments()
        with torch.cuda.stream(stream):
            s.step(S, mode)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = max(1, min(args.steps, 4))
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for _ in range(reps):
                s.step(S, mode)
            ev[1].record(stream)
        torch.cuda.synchronize(dev)
        ms = ev[0].elapsed_time(ev[1]) / reps
        rc = s.status()
        if rc != at.AT_OK:
            raise RuntimeError(f"system {name}: device status {rc}: {at.at_last_error()}")
        info = s.info()
        res[name] = {"value": npts * S / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_launch": ms, "ctas": info.ctas,
                     "stages": info.stages}
        if name == "free":
            res["moments_after"] = s.moments()
            res["moments_after_steps"] = S * (1 + reps)
        s.close()
    res["speedup_free_over_sync"] = res["free"]["value"] / res["sync"]["value"]
    bpu = nf * (2 * 4 + 18 * 4 / sub[0])
    peak, src = hbm_peak()
    res["roofline"] = {"bound": "hbm", "algorithmic_bytes_per_update": bpu, "achieved": res["free"]["value"] * bpu,
                       "peak": peak, "unit": "GB/s", "frac": res["free"]["value"] * bpu / peak, "peak_source": src}
    import oracle
    nb = 64
    qb = np.stack([0.5 * W.u0_spectral3d(nb, seed=4 + f, kmax=16) for f in range(nf)])
    kb = [0.1, 0.1, 0.1, 0.05, 0.2]
    dtb = W.dt_rule(qb[:3].reshape(-1), 2 * np.pi / nb, max(kb), dim=3)
    s = at.System3D((nb, nb, nb), sub, L, kb, dtb, dtype="f32", seed=5, device=dev.index)
    s.set_state(torch.from_numpy(qb.ravel()).to(dev))
    s.step(30, at.AT_SEEDED)
    g = s.state().double().cpu().numpy().reshape(qb.shape)
    s.close()
    ref, _ = oracle.run3d_system(qb, kappa=kb, P=(4, 4, 4), L=L, dt=dtb, n_steps=30, delay_mode=oracle.SEEDED, seed=5)
    res["err_vs_fp64_oracle"] = {"rel_linf_per_field": [float(np.max(np.abs(g[f] - ref[f])) / np.max(np.abs(ref[f])))
                                                        for f in range(nf)], "box": [nb] * 3, "steps": 30}
    return res


def reference_arm(args, ws, rank, pg):
    """--impl reference: the CPU oracle timed on this workload on every host
    core (OpenMP over subdomains), bounded sample per step."""
    cfg = W.config(WORKLOAD)
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = oracle.threads(os.cpu_count() or 1)
    N, P, M = cfg["N"], cfg["P"], cfg["N"] // cfg["P"]
    nsub = 4096
    full = W.initial_field(cfg)
    _, dx = W.grid(N)
    dt = W.dt_rule(full, dx, cfg["nu"])
    u0 = np.ascontiguousarray(full[:nsub * M])
    del full
    steps_per = max(1, args.time_steps // 100)
    kw = dict(N=N, P=P, order=cfg["order"], L=cfg["L"], nu=cfg["nu"], dt=dt, n_steps=steps_per,
              forcing_amp=cfg["forcing_amp"], delay_mode=oracle.SEEDED, seed=cfg["seed"], p_lo=0, p_count=nsub)
    for _ in range(args.warmup):
        oracle.run(u0, **kw)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(u0, **kw)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    upd = nsub * M * steps_per * args.steps
    val = upd / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "P": P, "order": cfg["order"], "L": cfg["L"],
                   "sample": f"{nsub} subdomains ({nsub * M} points) x {steps_per} steps per bench step"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{nsub * M} points x {steps_per} seeded steps per bench step, "
                                   f"OpenMP over subdomains on {cores} threads"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def fma_peaks(at):
    """Measured FMA rates of this GPU (FP64 and FP32), FMAs per second."""
    return {"f64": at.at_fma_peak(at.AT_F64, 1500), "f32": at.at_fma_peak(at.AT_F32, 100000)}


def timing_stats(per_ms):
    q = statistics.quantiles(per_ms, n=4) if len(per_ms) >= 2 else [per_ms[0]] * 3
    return {"median": statistics.median(per_ms), "q1": q[0], "q3": q[2], "launches": len(per_ms)}


def gpu_arm(args, ws, rank, local, pg):
    import torch

    import paper_1911_05769_gb300 as at
    from paper_1911_05769_gb300 import build as atbuild
    if rank == 0:
        atbuild.build()
    if pg is not None:
        pg.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = W.config(WORKLOAD)
    if args.N:
        cfg = dict(cfg, N=args.N, P=args.N // (cfg["N"] // cfg["P"]))
    if args.M:
        cfg = dict(cfg, P=cfg["N"] // args.M)
    if args.order:
        cfg = dict(cfg, order=args.order)
    if args.forcing >= 0:
        cfg = dict(cfg, forcing_amp=args.forcing)
    N, P, order, L, nu, A = cfg["N"], cfg["P"], cfg["order"], cfg["L"], cfg["nu"], cfg["forcing_amp"]
    u0 = W.initial_field(cfg)
    _, dx = W.grid(N)
    dt = W.dt_rule(u0, dx, nu)
    S = args.time_steps
    tdt = torch.float32 if args.dtype == "f32" else torch.float64
    wbytes = 4 if args.dtype == "f32" else 8
    u0_dev = torch.from_numpy(u0).to(device=dev, dtype=tdt)
    stream = torch.cuda.Stream(device=dev)

    spp = L + 1 if args.spp < 0 else args.spp

    def make(dtype=args.dtype, sb=spp, flags=0):
        return at.Solver(N, P, order, L, nu, dt, dtype=dtype, forcing_amp=A, seed=cfg["seed"], stream=stream,
                         device=local, max_ctas=args.ctas, stages=args.stages, steps_per_pass=sb, flags=flags)

    def barrier():
        if pg is not None:
            pg.barrier()

    def max_over_ranks_here(x):
        return max_over_ranks(pg, x, dev)

    def timed_arm(mode, sb, steps, warmup, time_steps, dtype=args.dtype, clocks=None, flags=0):
        s = make(dtype, sb, flags)
        s.set_state(u0_dev if dtype == args.dtype else u0_dev.to(torch.float64 if dtype == "f64" else torch.float32))
        for _ in range(warmup):
            s.step(time_steps, mode)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        if clocks:
            clocks.start()
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for i in range(steps):
                s.step(time_steps, mode)
                ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        clk = clocks.stop() if clocks else None
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        tot = ev[0].elapsed_time(ev[steps])
        rc = s.status()
        if rc != at.AT_OK:
            raise RuntimeError(f"{mode}: device status {rc}: {at.at_last_error()}")
        info = s.info()
        hist, m1, m2 = s.delay_stats()
        s.close()
        return dict(total_ms=max_over_ranks_here(tot), launch_ms=per, info=info, m1=m1, m2=m2, clocks=clk)

    clocks = Clocks(local)
    # the arms, timed back to back: free-running in passes of L+1 levels (the
    # headline), synchronous with a barrier every step, synchronous in passes
    # of L+1 levels (ghost cells), seeded delays, free-running one level per pass
    arm_defs = [("free_blocked", at.AT_FREE, spp), ("sync", at.AT_SYNC, 0), ("sync_blocked", at.AT_SYNC, spp),
                ("seeded", at.AT_SEEDED, 0), ("free", at.AT_FREE, 0)]
    want = set(args.arms.split(","))
    runs = {}
    for name, mode, sb in arm_defs:
        if name == "free_blocked" or name in want or "all" in want:
            runs[name] = timed_arm(mode, sb, args.steps, args.warmup, S, clocks=clocks if name == "free_blocked" else None)
    head = runs["free_blocked"]

    upd_per_step = N * S

    def gpts(r, steps=args.steps, per=upd_per_step):
        return whole_job_rate(ws, per * steps, r["total_ms"] * 1e-3)

    value = gpts(head)
    ms_per_step = head["total_ms"] / args.steps

    # roofline of the stepper kernel: algorithmic bytes per launch / launch time
    M, R, s_lev = N // P, order // 2, order // 2 + 1
    # one HBM read and write of the state per pass of `spp` levels, plus the
    # ring values a subdomain publishes (every level) and reads (every pass)
    bytes_per_update = (2 * wbytes + 2 * R * s_lev * wbytes / M) / max(1, spp) + 2 * R * wbytes / M
    alg_bytes = bytes_per_update * upd_per_step
    launch_s = statistics.mean(head["launch_ms"]) * 1e-3
    achieved = alg_bytes / launch_s / 1e9
    peak, peak_src = hbm_peak()
    traffic, traffic_steps = ncu_traffic()
    if traffic is not None and traffic_steps:
        traffic = traffic * S / traffic_steps
    # FP32 operations per update of the order-4 forced stencil (FMA = one op):
    # first difference 3, second difference 4, viscous/advective terms 3,
    # forcing 2, Euler update 1
    ops_per_update = 13
    peaks = fma_peaks(at)
    clk = (head["clocks"] or {}).get("sm_mhz") or 2070.0
    sms = head["info"].sm_count
    alu_peak = peaks["f32"] / 1e12
    alu_achieved = ops_per_update * upd_per_step / launch_s / 1e12
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_source": peak_src,
            "kernel": f"at_stepper<{'float' if wbytes == 4 else 'double'},4>",
            "algorithmic_bytes_per_update": bytes_per_update,
            "effective_one_pass": {"achieved": upd_per_step * 2 * wbytes / launch_s / 1e9, "unit": "GB/s",
                                   "frac": upd_per_step * 2 * wbytes / launch_s / 1e9 / peak,
                                   "note": "updates/s x 2 words: the HBM bytes a one-pass-per-step kernel would need"},
            "alu": None if wbytes != 4 else {
                "achieved": alu_achieved, "peak": alu_peak, "unit": "T FMA-pipe ops/s (FP32, FMA = 1 op)",
                "frac": alu_achieved / alu_peak, "ops_per_update": ops_per_update,
                "peak_source": "measured: at_fma_peak (FP32 FMA chains, all SMs)"}}

    def arm_line(name):
        r = runs.get(name)
        if r is None:
            return None
        return {"value": gpts(r), "ms_per_step": r["total_ms"] / args.steps, "ms_per_launch": timing_stats(r["launch_ms"]),
                "mean_k": r["m1"], "mean_k2": r["m2"], "steps_per_pass": r["info"].steps_per_pass if name in (
                    "free_blocked", "sync_blocked") else 1}

    at_vs_sync = {n: arm_line(n) for n, _, _ in arm_defs}
    if runs.get("sync"):
        at_vs_sync["speedup_free_over_sync"] = value / gpts(runs["sync"])
    if runs.get("sync_blocked"):
        at_vs_sync["speedup_free_over_sync_blocked"] = value / gpts(runs["sync_blocked"])
    if runs.get("free") and runs.get("sync"):
        at_vs_sync["speedup_free_unblocked_over_sync"] = gpts(runs["free"]) / gpts(runs["sync"])
    at_vs_sync["baselines"] = ("sync: a grid barrier every step, one HBM pass per step; sync_blocked: a grid barrier "
                               "every L+1 steps, one HBM pass per L+1 steps (ghost cells recomputed, bit for bit the "
                               "sync result); free_blocked: the headline, no barrier, passes of L+1 levels")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "ms_per_step_median": timing_stats(head["launch_ms"])["median"],
        "ms_per_step_q1": timing_stats(head["launch_ms"])["q1"], "ms_per_step_q3": timing_stats(head["launch_ms"])["q3"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "P": P, "M": M, "order": order, "L": L, "nu": nu,
                   "forcing_amp": A, "dt": dt, "time_steps_per_step": S, "mode": "free",
                   "steps_per_pass": spp,
                   "ctas": head["info"].ctas, "stages": head["info"].stages,
                   "l2": f"inputs larger than L2: state {N * wbytes / 2**20:.0f} MiB updated in place (no flush)",
                   "parallelism": "replicas" if ws > 1 else "single-gpu"},
        "gpu_launches": args.steps,
        "gpu_launches_note": "one at_stepper launch per bench step in the headline arm",
        "roofline": roof,
        "clocks": head["clocks"],
        "fma_peak": {"f64_tfma_per_s": peaks["f64"] / 1e12, "f32_tfma_per_s": peaks["f32"] / 1e12,
                     "sm_mhz_bench": clk, "note": "at_fma_peak: independent FMA chains on every SM, CUDA events"},
        "at_vs_sync": at_vs_sync,
    }

    if not args.no_extra:
        # e2e: host buffers through the C ABI, copies inside the timed region
        s = make()
        host_in = torch.from_numpy(u0).to(tdt).pin_memory()
        host_out = torch.empty(N, dtype=tdt).pin_memory()
        for _ in range(1):
            at.at_set_state(s.h, host_in.data_ptr())
            s.step(S, at.AT_FREE)
            at.at_state(s.h, host_out.data_ptr())
        e2e_steps = max(1, min(args.steps, 5))
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            rc = (at.at_set_state(s.h, host_in.data_ptr()), at.at_step(s.h, S, at.AT_FREE, None),
                  at.at_state(s.h, host_out.data_ptr()))
            if any(rc):
                raise RuntimeError(f"e2e: {rc} {at.at_last_error()}")
        el = max_over_ranks_here(time.perf_counter() - t0)
        s.close()
        line["e2e"] = {"value": whole_job_rate(ws, upd_per_step * e2e_steps, el), "unit": UNIT,
                       "h2d_bytes_per_step": N * wbytes, "d2h_bytes_per_step": N * wbytes,
                       "steps": e2e_steps}
        # FP64 state (FP64 arithmetic) on the same workload, fewer time steps;
        # bound by the FP64 FMA rate
        S64 = max(1, S // 10)
        f64 = timed_arm(at.AT_FREE, spp, 3, 2, S64, dtype="f64")
        v64 = whole_job_rate(ws, N * S64 * 3, f64["total_ms"] * 1e-3)
        ops64 = ops_per_update * v64 * 1e9 / 1e12
        line["f64"] = {"value": v64, "unit": UNIT, "time_steps_per_step": S64,
                       "roofline": {"bound": "fp64 alu", "achieved": ops64, "peak": peaks["f64"] / 1e12,
                                    "unit": "T FP64 FMA-pipe ops/s (FMA = 1 op)", "frac": ops64 / (peaks["f64"] / 1e12),
                                    "ops_per_update": ops_per_update,
                                    "peak_source": "measured: at_fma_peak (FP64 FMA chains, all SMs)",
                                    "hbm_frac": v64 * (2 * 8 / max(1, spp)) / peak}}
        if args.dtype == "f32":
            # the FP32 precision variants in the headline configuration
            for key, fl, note in (
                    ("compensated", at.AT_FLAG_COMPENSATED,
                     "FP32 hi + lo words per point, word-by-word stencil differences, two-sum updates; 2 CTAs per SM"),
                    ("viscous_fp64", at.AT_FLAG_VISCOUS_FP64,
                     "FP32 state, viscous term nu dt D2 formed and added in FP64 (forced on)")):
                r = timed_arm(at.AT_FREE, spp, 3, 2, S, flags=fl)
                line[key] = {"value": gpts(r, steps=3), "unit": UNIT, "mode": "free, passes of L+1", "note": note}
        if rank == 0 and ws == 1:
            line["cpu_baseline"] = cpu_baseline(args, u0, dt, cfg)
            line["accuracy"] = accuracy_legs(args, at, torch, stream, local, cfg, u0, u0_dev, dt, spp)
            for key, arm in (("compensated", "free_blocked_compensated"), ("viscous_fp64", "free_blocked_viscous_fp64")):
                if key in line and arm in line["accuracy"]:
                    line[key]["err_vs_fp64_oracle"] = line["accuracy"][arm]["rel_linf_vs_oracle_same_delays"]
        # the latency-bound case: N = 4096, P = 16 subdomains of 256 points,
        # order 2, L = 2, FP64 (one PE per subdomain, four CTAs), AT vs barrier
        line["small_config"] = small_config(args, at, torch, dev, stream)
        if rank == 0 and ws == 1:
            line["ensemble"] = ensemble_config(args, at, torch, dev, stream)
            line["adjoint"] = adjoint_config(args, at, torch, dev)
            line["burgers3d"] = config3d(args, at, torch, dev)
            line["system3d"] = config_system(args, at, torch, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)


def accuracy_legs(args, at, torch, stream, local, cfg, u0, u0_dev, dt, spp):
    """Equal error: every arm advanced 100 steps from the same state on the
    GPU, compared on a window of the workload's subdomains (away from its
    ends) with the FP64 oracle -- with the arm's own delays (parity) and with
    the synchronous run (accuracy), and the AT arms against the envelope
    2 |u(k=L) - u_sync| + 10 eps max|u_sync| (any admissible delay pattern)."""
    N, P, order, L, nu, A = cfg["N"], cfg["P"], cfg["order"], cfg["L"], cfg["nu"], cfg["forcing_amp"]
    M = N // P
    steps = args.cpu_sample_steps
    nsub = min(args.cpu_sample_subdomains, P)
    arms = [("free_blocked", at.AT_FREE, spp, 0), ("free", at.AT_FREE, 0, 0), ("seeded", at.AT_SEEDED, 0, 0),
            ("sync", at.AT_SYNC, 0, 0), ("sync_blocked", at.AT_SYNC, spp, 0)]
    if args.dtype == "f32":
        arms += [("free_blocked_compensated", at.AT_FREE, spp, at.AT_FLAG_COMPENSATED),
                 ("free_blocked_viscous_fp64", at.AT_FREE, spp, at.AT_FLAG_VISCOUS_FP64)]
    got, recs = {}, {}
    for name, mode, sb, flags in arms:
        s = at.Solver(N, P, order, L, nu, dt, dtype=args.dtype, forcing_amp=A, seed=cfg["seed"], stream=stream,
                      device=local, steps_per_pass=sb, flags=flags)
        s.set_state(u0_dev)
        d = torch.full((steps, P, 2), -1, dtype=torch.int8, device=u0_dev.device)
        s.step(steps, mode, d)
        u = s.state().double().cpu().numpy()[:nsub * M]
        if flags & at.AT_FLAG_COMPENSATED:
            u = u + s.state_error().double().cpu().numpy()[:nsub * M]
        got[name] = u
        if mode == at.AT_FREE:
            recs[name] = d.cpu().numpy()
        s.close()
    ref, nsub, steps = window_oracles(args, u0, dt, cfg, recs)
    cut = (order // 2) * steps + M
    sl = slice(cut, nsub * M - cut)
    scale = float(np.max(np.abs(ref["sync"][sl])))
    eps = float(np.finfo(np.float32 if args.dtype == "f32" else np.float64).eps)
    env = 2.0 * float(np.max(np.abs(ref["k_eq_L"][sl] - ref["sync"][sl]))) + 10.0 * eps * scale
    out = {"window": f"{nsub} subdomains ({nsub * M} points), {steps} steps from the same state, "
                     f"{nsub * M - 2 * cut} points compared", "dtype": args.dtype,
           "envelope_abs": env, "k_eq_L_vs_sync_rel_linf": float(np.max(np.abs(ref["k_eq_L"][sl] - ref["sync"][sl]))) / scale}
    for name, mode, sb, flags in arms:
        own = ref[name] if name in recs else (ref["sync"] if mode == at.AT_SYNC else ref["seeded"])
        e_own = float(np.max(np.abs(got[name][sl] - own[sl]))) / scale
        d_sync = float(np.max(np.abs(got[name][sl] - ref["sync"][sl])))
        # the envelope bounds any admissible free-running result
        out[name] = {"rel_linf_vs_oracle_same_delays": e_own, "rel_linf_vs_fp64_sync": d_sync / scale,
                     "within_envelope": bool(d_sync <= env) if mode == at.AT_FREE else None}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        # the oracle runs on rank 0 only; other ranks exit without work
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        reference_arm(args, ws, rank, None)
        return
    ws, rank, local, pg = dist_setup(args)
    if args.only_system:
        import torch

        import paper_1911_05769_gb300 as at
        from paper_1911_05769_gb300 import build as atbuild
        atbuild.build()
        torch.cuda.set_device(local)
        print(json.dumps(config_system(args, at, torch, torch.device("cuda", local))), flush=True)
        return
    if args.only_3d:
        import torch

        import paper_1911_05769_gb300 as at
        from paper_1911_05769_gb300 import build as atbuild
        atbuild.build()
        torch.cuda.set_device(local)
        print(json.dumps(config3d(args, at, torch, torch.device("cuda", local))), flush=True)
        return
    if args.adjoint_only:
        import torch

        import paper_1911_05769_gb300 as at
        from paper_1911_05769_gb300 import build as atbuild
        atbuild.build()
        torch.cuda.set_device(local)
        print(json.dumps(adjoint_config(args, at, torch, torch.device("cuda", local))), flush=True)
        return
    if args.ensemble_only:
        import torch

        import paper_1911_05769_gb300 as at
        from paper_1911_05769_gb300 import build as atbuild
        atbuild.build()
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        print(json.dumps(ensemble_config(args, at, torch, dev, torch.cuda.Stream(device=dev))), flush=True)
        return
    gpu_arm(args, ws, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
