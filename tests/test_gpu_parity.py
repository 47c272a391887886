"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: relative L-inf <= 1e-12 for FP64 state, <= 1e-5 for FP32 state; delays
(integers) bit-exact.  FP32 cases keep the step count where round-to-nearest
FP32 state stays within 1e-5 of the FP64 result (a few hundred steps at these
sizes; the drift is a property of FP32 storage, not of the method).
"""
import numpy as np
import pytest

import at_workloads as W
import oracle
from gpu_util import TOL, gpu_run, oracle_run, rel_linf

pytestmark = pytest.mark.gpu


def _setup(N, nu, kind="two_modes", seed=2):
    u0 = W.u0_two_modes(N) if kind == "two_modes" else W.u0_fourier(N, modes=64, seed=seed)
    _, dx = W.grid(N)
    return u0, W.dt_rule(u0, dx, nu)


def test_burgers1d_n4096_seeded_fp64(require_gpu):
    """N=4096, P=16, order 2, L=2, seeded delays (seed 1), 1000 steps, FP64."""
    from paper_1911_05769_gb300 import AT_SEEDED
    cfg = W.config("burgers1d_n4096")
    u0 = W.initial_field(cfg)
    _, dx = W.grid(cfg["N"])
    dt = W.dt_rule(u0, dx, cfg["nu"])
    kw = dict(P=cfg["P"], order=cfg["order"], L=cfg["L"], nu=cfg["nu"], dt=dt, steps=cfg["n_steps"])
    g = gpu_run(u0, mode=AT_SEEDED, seed=cfg["seed"], record=True, **kw)
    ref, hist, k = oracle_run(u0, mode="seeded", seed=cfg["seed"], want_k=True, **kw)
    assert rel_linf(g["u"], ref) <= TOL["f64"]
    assert np.array_equal(g["rec"], k)          # delays: bit-exact
    assert np.array_equal(g["hist"], hist)
    assert hist[1:].sum() > 0


CASES = [
    # dtype, order, L, P, M, max_ctas, forcing, steps, stages
    ("f64", 4, 3, 148, 256, 10, 0.1, 300, 0),     # ragged CTA partition (14/15 subdomains)
    ("f64", 2, 2, 37, 1020, 5, 0.0, 200, 0),      # M/4 = 255 groups: a ragged last row of lanes
    ("f64", 4, 1, 8, 1024, 3, 0.1, 150, 0),       # largest tile, FP64
    ("f32", 4, 3, 64, 1024, 0, 0.1, 200, 0),      # forced order-4 subdomains of 1024 points
    ("f32", 2, 2, 16, 256, 4, 0.0, 200, 0),
    ("f32", 4, 3, 3, 1024, 0, 0.1, 100, 0),       # largest FP32 tile, one subdomain per CTA
    ("f64", 2, 0, 32, 64, 7, 0.0, 300, 0),        # L = 0
    ("f64", 2, 16, 64, 32, 8, 0.0, 200, 0),       # L = 16 (largest), see below
    ("f64", 2, 2, 1, 256, 0, 0.0, 200, 0),        # one subdomain, its own neighbour
    ("f64", 4, 3, 40, 4, 6, 0.0, 200, 0),         # M = 4: one group per tile
    ("f64", 4, 3, 96, 128, 4, 0.1, 200, 4),       # fewest stages (one per consumer warp)
    ("f64", 2, 3, 96, 132, 4, 0.1, 200, 5),       # stages not a multiple of the warps
    ("f32", 4, 2, 300, 512, 0, 0.1, 150, 0),      # 300 subdomains over all SMs, ragged
]


@pytest.mark.parametrize("dtype,order,L,P,M,max_ctas,forcing,steps,stages", CASES)
def test_seeded_parity(require_gpu, dtype, order, L, P, M, max_ctas, forcing, steps, stages):
    from paper_1911_05769_gb300 import AT_SEEDED
    N = P * M
    u0, dt = _setup(N, 0.02, kind="fourier" if N >= 256 else "two_modes")
    # L = 16 runs at order 2: with order 4 the quadratic extrapolation weights
    # reach 153 at k = 16 and the problem itself amplifies a 1-ulp change of u0
    # to ~4e-9 after 200 steps, so no differently rounded FP64 code can meet 1e-12.
    kw = dict(P=P, order=order, L=L, nu=0.02, dt=dt, steps=steps, seed=1234 + P, forcing=forcing)
    g = gpu_run(u0, dtype=dtype, mode=AT_SEEDED, max_ctas=max_ctas, stages=stages, record=True, **kw)
    ref, hist, k = oracle_run(u0, mode="seeded", want_k=True, **kw)
    assert rel_linf(g["u"], ref) <= TOL[dtype]
    assert np.array_equal(g["rec"], k)
    assert np.array_equal(g["hist"], hist)


@pytest.mark.parametrize("dtype,order,max_ctas", [("f64", 2, 0), ("f64", 4, 5), ("f32", 4, 3), ("f64", 4, 1)])
def test_sync_parity(require_gpu, dtype, order, max_ctas):
    """AT_SYNC (grid barrier every step, Algorithm 1) against the synchronous oracle."""
    from paper_1911_05769_gb300 import AT_SYNC
    N, P = 64 * 128, 64
    u0, dt = _setup(N, 0.02, kind="fourier")
    kw = dict(P=P, order=order, L=2, nu=0.02, dt=dt, steps=200 if dtype == "f32" else 400, forcing=0.1)
    g = gpu_run(u0, dtype=dtype, mode=AT_SYNC, max_ctas=max_ctas, record=True, **kw)
    ref, hist = oracle_run(u0, mode="sync", **kw)
    assert rel_linf(g["u"], ref) <= TOL[dtype]
    assert np.all(g["rec"] == 0) and g["hist"][0] == hist[0] and g["hist"][1:].sum() == 0


def test_zero_delay_modes_are_bitwise_synchronous(require_gpu):
    """Sec. 3.2: k = 0 gives the standard scheme -- on the GPU, SEEDED with
    L = 0 and REPLAY of zeros reproduce AT_SYNC bit for bit."""
    from paper_1911_05769_gb300 import AT_REPLAY, AT_SEEDED, AT_SYNC
    N, P = 32 * 256, 32
    u0, dt = _setup(N, 0.02, kind="fourier")
    kw = dict(P=P, order=4, nu=0.02, dt=dt, steps=300, forcing=0.1, max_ctas=6)
    a = gpu_run(u0, L=0, mode=AT_SYNC, **kw)["u"]
    b = gpu_run(u0, L=0, mode=AT_SEEDED, seed=3, **kw)["u"]
    c = gpu_run(u0, L=2, mode=AT_REPLAY, delays=np.zeros((300, P, 2), np.int8), **kw)["u"]
    assert np.array_equal(a, b) and np.array_equal(a, c)


@pytest.mark.parametrize("dtype,order", [("f64", 2), ("f64", 4), ("f32", 4)])
def test_replay_parity(require_gpu, dtype, order):
    from paper_1911_05769_gb300 import AT_REPLAY
    N, P, L, steps = 48 * 256, 48, 3, 200
    u0, dt = _setup(N, 0.02, kind="fourier")
    d = W.random_delays(steps, P, L, seed=77)
    kw = dict(P=P, order=order, L=L, nu=0.02, dt=dt, steps=steps, forcing=0.1)
    g = gpu_run(u0, dtype=dtype, mode=AT_REPLAY, delays=d, max_ctas=5, **kw)
    ref, hist = oracle_run(u0, mode="replay", delays=d, **kw)
    assert rel_linf(g["u"], ref) <= TOL[dtype]
    assert np.array_equal(g["hist"], hist)


@pytest.mark.parametrize("dtype,max_ctas", [("f64", 0), ("f64", 7), ("f32", 0)])
def test_free_running_replays_exactly(require_gpu, dtype, max_ctas):
    """Free-running delays have many correct results (c15): the GPU records
    the delays it used, the oracle replays them and must agree to the bar;
    every recorded delay lies in 0..L."""
    from paper_1911_05769_gb300 import AT_FREE
    N, P, L, steps = 256 * 128, 256, 3, 300 if dtype == "f64" else 150
    u0, dt = _setup(N, 0.02, kind="fourier")
    kw = dict(P=P, order=4, L=L, nu=0.02, dt=dt, steps=steps, forcing=0.1)
    g = gpu_run(u0, dtype=dtype, mode=AT_FREE, max_ctas=max_ctas, record=True, **kw)
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= L
    assert g["hist"].sum() == steps * P * 2
    ref, hist = oracle_run(u0, mode="replay", delays=rec, **kw)
    assert rel_linf(g["u"], ref) <= TOL[dtype]
    assert np.array_equal(g["hist"], hist)


def test_free_running_within_asynchrony_envelope(require_gpu):
    """FREE results stay within the error the scheme makes with the largest
    admissible delay everywhere (k = L), measured from the synchronous run."""
    from paper_1911_05769_gb300 import AT_FREE
    N, P, L, steps = 128 * 128, 128, 3, 400
    u0, dt = _setup(N, 0.02, kind="fourier")
    kw = dict(P=P, order=2, L=L, nu=0.02, dt=dt, steps=steps)
    g = gpu_run(u0, mode=AT_FREE, max_ctas=9, **kw)["u"]
    sync, _ = oracle_run(u0, mode="sync", **kw)
    worst, _ = oracle_run(u0, mode="replay", delays=np.full((steps, P, 2), L, np.int8), **kw)
    env = 2.0 * np.max(np.abs(worst - sync)) + 10 * np.finfo(np.float64).eps * np.max(np.abs(sync))
    assert np.max(np.abs(g - sync)) <= env


def test_calls_continue_one_another(require_gpu):
    """Several at_step calls equal one long run (ring, flags and the step
    counter persist across launches), in seeded and in replayed mode."""
    from paper_1911_05769_gb300 import AT_REPLAY, AT_SEEDED, AT_SYNC
    N, P, L, steps = 40 * 256, 40, 2, 300
    u0, dt = _setup(N, 0.02, kind="fourier")
    kw = dict(P=P, order=4, L=L, nu=0.02, dt=dt, steps=steps, forcing=0.1)
    g = gpu_run(u0, mode=AT_SEEDED, seed=9, max_ctas=6, calls=[100, 37, 1, 162], **kw)
    ref, _ = oracle_run(u0, mode="seeded", seed=9, **kw)
    assert rel_linf(g["u"], ref) <= TOL["f64"]
    d = W.random_delays(steps, P, L, seed=5)
    g = gpu_run(u0, mode=AT_REPLAY, delays=d, max_ctas=6, calls=[150, 150], **kw)
    ref, _ = oracle_run(u0, mode="replay", delays=d, **kw)
    assert rel_linf(g["u"], ref) <= TOL["f64"]
    # a synchronous call in between: the ring stays consistent
    g1 = gpu_run(u0, mode=AT_SYNC, max_ctas=6, calls=[300], **kw)["u"]
    ref, _ = oracle_run(u0, mode="sync", **kw)
    assert rel_linf(g1, ref) <= TOL["f64"]


def test_per_subdomain_delay_draw(require_gpu):
    from paper_1911_05769_gb300 import AT_FLAG_PER_SUBDOMAIN_DELAY, AT_SEEDED
    N, P, L, steps = 32 * 128, 32, 2, 200
    u0, dt = _setup(N, 0.02, kind="fourier")
    kw = dict(P=P, order=2, L=L, nu=0.02, dt=dt, steps=steps, seed=21)
    g = gpu_run(u0, mode=AT_SEEDED, flags=AT_FLAG_PER_SUBDOMAIN_DELAY, record=True, max_ctas=4, **kw)
    ref, _, k = oracle_run(u0, mode="seeded", per_subdomain=True, want_k=True, **kw)
    assert np.array_equal(g["rec"], k)
    assert rel_linf(g["u"], ref) <= TOL["f64"]


def test_empty_step_is_a_no_op(require_gpu):
    from paper_1911_05769_gb300 import AT_SEEDED
    N, P = 16 * 64, 16
    u0, dt = _setup(N, 0.02)
    g = gpu_run(u0, P=P, order=2, L=1, nu=0.02, dt=dt, steps=0, calls=[0], mode=AT_SEEDED)
    assert np.array_equal(g["u"], u0)


BLOCKED = [
    # dtype, order, L, steps_per_pass, P, M, max_ctas, steps, calls
    ("f64", 4, 3, 4, 96, 256, 7, 300, None),
    ("f64", 2, 2, 3, 64, 128, 5, 301, [100, 1, 200]),
    ("f64", 4, 3, 2, 40, 1020, 3, 150, None),
    ("f32", 4, 3, 4, 256, 1024, 0, 200, None),
    ("f64", 2, 1, 2, 1, 256, 0, 120, None),        # one subdomain, its own neighbour
    ("f64", 4, 3, 4, 40, 4, 6, 100, [3, 97]),      # M = 4 (N = 160: a coarser grid is unstable for
                                                   # forward Euler itself at this CFL number)
]


@pytest.mark.parametrize("dtype,order,L,spp,P,M,max_ctas,steps,calls", BLOCKED)
def test_blocked_free_running_replays_exactly(require_gpu, dtype, order, L, spp, P, M, max_ctas, steps, calls):
    """Temporal blocking in free-running mode: a tile advances `spp` levels per
    pass with halos extrapolated from the levels available at the start of the
    pass (delay k0 + i at inner step i).  The recorded delays, replayed by the
    oracle, reproduce the result to the bar; every delay stays within L."""
    from paper_1911_05769_gb300 import AT_FREE
    N = P * M
    u0, dt = _setup(N, 0.02, kind="fourier" if N >= 256 else "two_modes")
    kw = dict(P=P, order=order, L=L, nu=0.02, dt=dt, steps=steps, forcing=0.1)
    g = gpu_run(u0, dtype=dtype, mode=AT_FREE, max_ctas=max_ctas, record=True, calls=calls,
                steps_per_pass=spp, **kw)
    rec = g["rec"]
    assert rec.min() >= 0 and rec.max() <= L
    assert g["hist"].sum() == steps * P * 2
    ref, hist = oracle_run(u0, mode="replay", delays=rec, **kw)
    assert rel_linf(g["u"], ref) <= TOL[dtype]
    assert np.array_equal(g["hist"], hist)
    if spp > 1 and calls is None:
        assert rec[:, :, :].max() >= 1      # the blocking did create delays


def test_blocked_passes_of_L_plus_1_are_deterministic(require_gpu):
    """With passes of L+1 levels every face must wait for level n exactly, so
    the delays are fixed by the pass structure: single levels while n < s-1,
    then k = (n - (s-1)) mod (L+1) within each full pass."""
    from paper_1911_05769_gb300 import AT_FREE
    N, P, L, order, steps = 64 * 256, 64, 3, 4, 2 + 4 * 50
    s_lev = order // 2 + 1
    u0, dt = _setup(N, 0.02, kind="fourier")
    g = gpu_run(u0, P=P, order=order, L=L, nu=0.02, dt=dt, steps=steps, mode=AT_FREE, max_ctas=6, record=True,
                steps_per_pass=L + 1)
    n = np.arange(steps)
    want = np.where(n < s_lev - 1, 0, (n - (s_lev - 1)) % (L + 1)).astype(np.int8)
    assert np.array_equal(g["rec"], np.broadcast_to(want[:, None, None], g["rec"].shape))


@pytest.mark.parametrize("stages", [2, 3, 4])
@pytest.mark.parametrize("per_pe,calls", [(1, None), (2, [37, 83]), (5, None), (9, [1, 119])])
def test_alternating_sweep_turns(require_gpu, stages, per_pe, calls):
    """Blocked free-running passes sweep each element's subdomains forth and
    back; the tile at a turn continues in registers and the tiles after it are
    loaded no earlier than their last write-back.  Every tile-buffer count
    and run length (1: every tile a turn; 2: every other tile) replays exactly
    in the oracle, also across calls of odd lengths."""
    from paper_1911_05769_gb300 import AT_FREE
    P, M, L = 8 * per_pe, 256, 3
    u0, dt = _setup(P * M, 0.02, kind="fourier")
    kw = dict(P=P, order=4, L=L, nu=0.02, dt=dt, steps=120, forcing=0.1)
    g = gpu_run(u0, mode=AT_FREE, max_ctas=2, stages=stages, record=True, calls=calls, steps_per_pass=L + 1, **kw)
    ref, hist = oracle_run(u0, mode="replay", delays=g["rec"], **kw)
    assert g["info"].ctas == 2
    assert rel_linf(g["u"], ref) <= TOL["f64"]
    assert np.array_equal(g["hist"], hist)


@pytest.mark.parametrize("per_pe", [1, 2, 3])
@pytest.mark.parametrize("mode_name", ["seeded", "free", "free_blocked", "sync"])
def test_subdomains_per_processing_element(require_gpu, per_pe, mode_name):
    """Each warp is one processing element owning a contiguous run of
    subdomains; 1, 2 and 3 subdomains per element exercise the edge-only, the
    no-prefetch and the prefetching halo paths.  Two CTAs = 8 elements."""
    import paper_1911_05769_gb300 as at
    P, M, L = 8 * per_pe, 128, 2
    N = P * M
    u0, dt = _setup(N, 0.02, kind="fourier")
    kw = dict(P=P, order=4, L=L, nu=0.02, dt=dt, steps=120, forcing=0.1)
    mode = {"seeded": at.AT_SEEDED, "free": at.AT_FREE, "free_blocked": at.AT_FREE, "sync": at.AT_SYNC}[mode_name]
    spp = L + 1 if mode_name == "free_blocked" else 0
    g = gpu_run(u0, mode=mode, seed=31, max_ctas=2, record=True, steps_per_pass=spp, **kw)
    if mode_name == "seeded":
        ref, hist, k = oracle_run(u0, mode="seeded", seed=31, want_k=True, **kw)
        assert np.array_equal(g["rec"], k)
    elif mode_name == "sync":
        ref, hist = oracle_run(u0, mode="sync", **kw)
    else:
        ref, hist = oracle_run(u0, mode="replay", delays=g["rec"], **kw)
    assert g["info"].ctas == 2
    assert rel_linf(g["u"], ref) <= TOL["f64"]
    assert np.array_equal(g["hist"], hist)


BLOCKED_SYNC = [
    # dtype, order, L, steps_per_pass, P, M, max_ctas, steps, calls, forcing, flags
    ("f64", 4, 3, 4, 96, 256, 7, 301, None, 0.1, 0),
    ("f32", 4, 3, 4, 256, 1024, 0, 200, [150, 50], 0.1, 0),
    ("f64", 2, 2, 3, 64, 128, 5, 200, [100, 1, 99], 0.0, 0),
    ("f32", 2, 7, 8, 48, 16, 4, 161, None, 0.1, 0),        # strips of 8 words, tiles of 16 points
    ("f64", 4, 3, 2, 40, 1020, 3, 150, None, 0.1, 0),      # ragged tiles (groups beyond 32 lanes)
    ("f64", 2, 1, 2, 1, 256, 0, 120, None, 0.0, 0),        # one subdomain, its own neighbour
    ("f64", 2, 2, 3, 3, 256, 0, 90, None, 0.1, 0),         # three subdomains on three PEs
    ("f64", 4, 3, 4, 40, 8, 6, 100, [3, 97], 0.1, 0),      # strips as wide as the tile
    ("f32", 4, 3, 4, 64, 256, 2, 120, None, 0.1, "v64"),   # FP64 viscous accumulation
]


@pytest.mark.parametrize("dtype,order,L,spp,P,M,max_ctas,steps,calls,forcing,flags", BLOCKED_SYNC)
def test_blocked_sync_is_bitwise_synchronous(require_gpu, dtype, order, L, spp, P, M, max_ctas, steps, calls,
                                             forcing, flags):
    """The blocked synchronous mode (AT_SYNC in passes of steps_per_pass
    levels, a grid barrier before each pass, every delay 0, the halo of each
    inner level recomputed from the neighbours' edge strips as ghost cells)
    equals the unblocked AT_SYNC run (a barrier every step) bit for bit, and
    the synchronous oracle to the bar."""
    from paper_1911_05769_gb300 import AT_FLAG_VISCOUS_FP64, AT_SYNC
    N = P * M
    u0, dt = _setup(N, 0.02, kind="fourier" if N >= 256 else "two_modes")
    fl = AT_FLAG_VISCOUS_FP64 if flags == "v64" else 0
    kw = dict(P=P, order=order, L=L, nu=0.02, dt=dt, steps=steps, forcing=forcing, flags=fl)
    blk = gpu_run(u0, dtype=dtype, mode=AT_SYNC, max_ctas=max_ctas, record=True, calls=calls, steps_per_pass=spp,
                  **kw)
    one = gpu_run(u0, dtype=dtype, mode=AT_SYNC, max_ctas=max_ctas, **kw)
    assert blk["info"].steps_per_pass == spp
    assert np.array_equal(blk["u"], one["u"]), rel_linf(blk["u"], one["u"])
    assert np.all(blk["rec"] == 0) and np.array_equal(blk["hist"], one["hist"])
    ref, _ = oracle_run(u0, mode="sync", P=P, order=order, L=L, nu=0.02, dt=dt, steps=steps, forcing=forcing)
    assert rel_linf(blk["u"], ref) <= TOL[dtype]


def test_blocked_sync_follows_other_modes(require_gpu):
    """A blocked synchronous launch takes its edge strips from the state it
    starts from, whatever ran before it: seeded, then blocked sync, then
    free-running blocked, then blocked sync again, against the oracle
    replaying the same delay sequence (zeros for the synchronous parts)."""
    import torch

    from paper_1911_05769_gb300 import AT_FREE, AT_SEEDED, AT_SYNC, Solver
    N, P, L, order = 64 * 256, 64, 3, 4
    u0, dt = _setup(N, 0.02, kind="fourier")
    s = Solver(N, P, order, L, 0.02, dt, dtype="f64", seed=9, forcing_amp=0.1, max_ctas=5, steps_per_pass=L + 1)
    s.set_state(torch.from_numpy(u0).cuda())
    parts = [(AT_SEEDED, 37), (AT_SYNC, 41), (AT_FREE, 30), (AT_SYNC, 22)]
    rec = []
    for mode, n in parts:
        d = torch.full((n, P, 2), -1, dtype=torch.int8, device="cuda")
        s.step(n, mode, d)
        rec.append(d.cpu().numpy())
    got = s.state().cpu().numpy()
    s.close()
    rec = np.concatenate(rec, axis=0)
    assert rec[37:78].max() == 0 and rec[108:].max() == 0
    ref, _ = oracle_run(u0, mode="replay", delays=rec, P=P, order=order, L=L, nu=0.02, dt=dt, steps=130,
                        forcing=0.1)
    assert rel_linf(got, ref) <= TOL["f64"]
