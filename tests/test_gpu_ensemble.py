"""Ensembles of independent problems in one persistent launch (at_create_batch):
each instance of the CUDA run against the oracle run of that instance alone
(its own grid, viscosity, time step, delay bound, seed and exact travelling-wave
boundary values), element by element.  Also the launch-shape autotuner and
replay of a captured CUDA graph."""
import numpy as np
import pytest

import at_workloads as W
import oracle
from gpu_util import TOL, gpu_ensemble_run, oracle_ensemble, rel_linf

pytestmark = pytest.mark.gpu


def small_ensemble(n_inst=7, seed=11, M=256, log2_n=(8.0, 11.5), periodic=()):
    inst = W.ensemble(n_inst=n_inst, seed=seed, M=M, log2_n=log2_n)
    for j in periodic:
        d = inst[j]
        x, dx = W.grid(d["n"], d["length"], d["origin"])
        d["bc"] = 0
        d["u0"] = 0.3 + 0.2 * np.sin(x) + 0.1 * np.sin(3 * x + 1)
        d["dt"] = W.dt_rule(d["u0"], dx, d["nu"])
    return inst


def split(u, offsets):
    return [u[offsets[j]:offsets[j + 1]] for j in range(len(offsets) - 1)]


def check_against_oracle(inst, res, *, M, order, steps, mode, dtype, delays=None, which=None):
    ref = oracle_ensemble(inst, M=M, order=order, steps=steps, mode=mode, delays=delays, which=which)
    parts = split(res["u"], res["offsets"])
    worst = 0.0
    for j, (u_ref, _) in ref.items():
        err = rel_linf(parts[j], u_ref)
        worst = max(worst, err)
        assert err <= TOL[dtype], (j, inst[j]["n"], inst[j]["L"], err)
    return ref, worst


def total_hist(ref, Lmax):
    h = np.zeros(Lmax + 1, dtype=np.int64)
    for _, hj in ref.values():
        h[:len(hj)] += hj
    return h


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("max_ctas", [2, 0])
def test_seeded_ensemble_matches_oracle(dtype, order, max_ctas):
    M = 256
    inst = small_ensemble(M=M)
    steps = 200
    res = gpu_ensemble_run(inst, M=M, order=order, steps=steps, dtype=dtype, max_ctas=max_ctas)
    ref, _ = check_against_oracle(inst, res, M=M, order=order, steps=steps, mode="seeded", dtype=dtype)
    Lmax = max(d["L"] for d in inst)
    assert res["info"].P == sum(d["n"] for d in inst) // M and res["info"].L == Lmax
    assert np.array_equal(res["hist"], total_hist(ref, Lmax))


@pytest.mark.parametrize("spp", [0, 4])
def test_free_ensemble_replays_in_oracle(spp):
    """Free-running delays (blocked passes with spp = 4: each processing
    element takes its passes no longer than its smallest L_j + 1) are recorded
    and replayed per instance by the oracle."""
    from paper_1911_05769_gb300 import AT_FREE
    M = 256
    inst = small_ensemble(M=M, seed=12)
    steps = 160
    res = gpu_ensemble_run(inst, M=M, order=2, steps=steps, dtype="f64", mode=AT_FREE, record=True, max_ctas=2,
                           steps_per_pass=spp)
    rec = res["rec"]
    p0 = 0
    for d in inst:
        Pj = d["n"] // M
        r = rec[:, p0:p0 + Pj, :]
        assert r.min() >= 0 and r.max() <= d["L"], (d["L"], r.min(), r.max())
        p0 += Pj
    check_against_oracle(inst, res, M=M, order=2, steps=steps, mode="replay", dtype="f64", delays=rec)


def test_replayed_ensemble_delays_match_oracle():
    from paper_1911_05769_gb300 import AT_REPLAY
    M = 256
    inst = small_ensemble(M=M, seed=13)
    steps = 150
    P = sum(d["n"] for d in inst) // M
    rng = np.random.default_rng(5)
    delays = np.empty((steps, P, 2), dtype=np.int8)
    p0 = 0
    for d in inst:
        Pj = d["n"] // M
        delays[:, p0:p0 + Pj, :] = rng.integers(0, d["L"] + 1, size=(steps, Pj, 2))
        p0 += Pj
    res = gpu_ensemble_run(inst, M=M, order=2, steps=steps, dtype="f64", mode=AT_REPLAY, delays=delays,
                           max_ctas=3)
    check_against_oracle(inst, res, M=M, order=2, steps=steps, mode="replay", dtype="f64", delays=delays)


@pytest.mark.parametrize("order", [2, 4])
def test_blocked_sync_ensemble_is_bitwise_synchronous(order):
    """Blocked synchronous passes in an ensemble (exact-boundary and periodic
    instances, one- and two-subdomain instances, uneven L_j): equal to the
    unblocked AT_SYNC run bit for bit; every PE takes the same passes
    whatever its L_j (the grid barrier before each pass needs that)."""
    from paper_1911_05769_gb300 import AT_SYNC
    M = 256
    inst = small_ensemble(M=M, seed=41 + order, log2_n=(8.0, 10.5), periodic=(0, 3))
    inst[0]["n"] = 256
    inst[3]["n"] = 512
    for j in (0, 3):
        d = inst[j]
        x, dx = W.grid(d["n"], d["length"], d["origin"])
        d["u0"] = 0.3 + 0.2 * np.sin(x) + 0.1 * np.sin(3 * x + 1)
        d["dt"] = W.dt_rule(d["u0"], dx, d["nu"])
    blk = gpu_ensemble_run(inst, M=M, order=order, steps=130, dtype="f64", mode=AT_SYNC, max_ctas=2,
                           steps_per_pass=4, calls=[70, 60])
    one = gpu_ensemble_run(inst, M=M, order=order, steps=130, dtype="f64", mode=AT_SYNC, max_ctas=2)
    assert blk["info"].steps_per_pass == 4
    assert np.array_equal(blk["u"], one["u"])
    check_against_oracle(inst, blk, M=M, order=order, steps=130, mode="sync", dtype="f64")


def test_sync_ensemble_matches_oracle():
    from paper_1911_05769_gb300 import AT_SYNC
    M = 256
    inst = small_ensemble(M=M, seed=14)
    res = gpu_ensemble_run(inst, M=M, order=2, steps=120, dtype="f64", mode=AT_SYNC, max_ctas=2)
    check_against_oracle(inst, res, M=M, order=2, steps=120, mode="sync", dtype="f64")


@pytest.mark.parametrize("max_ctas", [1, 2, 0])
def test_periodic_and_tiny_instances(max_ctas):
    """Periodic instances among exact-boundary ones, including one- and
    two-subdomain instances (a face whose neighbour is the subdomain itself,
    or the same neighbour on both faces)."""
    M = 256
    inst = small_ensemble(M=M, seed=15, log2_n=(8.0, 10.0), periodic=(0, 2, 3))
    inst[0]["n"] = 256                     # one subdomain, periodic: its own neighbour
    inst[2]["n"] = 512                     # two subdomains, periodic
    for j in (0, 2):
        d = inst[j]
        x, dx = W.grid(d["n"], d["length"], d["origin"])
        d["u0"] = 0.3 + 0.2 * np.sin(x)
        d["dt"] = W.dt_rule(d["u0"], dx, d["nu"])
    for mode in ("seeded", "free"):
        from paper_1911_05769_gb300 import AT_FREE, AT_SEEDED
        if mode == "seeded":
            res = gpu_ensemble_run(inst, M=M, order=2, steps=150, dtype="f64", mode=AT_SEEDED, max_ctas=max_ctas)
            check_against_oracle(inst, res, M=M, order=2, steps=150, mode="seeded", dtype="f64")
        else:
            res = gpu_ensemble_run(inst, M=M, order=2, steps=150, dtype="f64", mode=AT_FREE, record=True,
                                   max_ctas=max_ctas, steps_per_pass=2)
            check_against_oracle(inst, res, M=M, order=2, steps=150, mode="replay", dtype="f64",
                                 delays=res["rec"])


def test_partial_tiles_and_multiple_calls():
    """M = 192 (tiles that do not fill the last lane group), order 4, and one
    run split over several at_step calls equals one call bit for bit."""
    M = 192
    inst = small_ensemble(M=M, seed=16, log2_n=(8.5, 11.0))
    one = gpu_ensemble_run(inst, M=M, order=4, steps=180, dtype="f64", max_ctas=2)
    three = gpu_ensemble_run(inst, M=M, order=4, steps=180, dtype="f64", max_ctas=2, calls=[50, 70, 60])
    assert np.array_equal(one["u"], three["u"])
    assert np.array_equal(one["hist"], three["hist"])
    check_against_oracle(inst, one, M=M, order=4, steps=180, mode="seeded", dtype="f64")


def test_autotuner_keeps_results_exact():
    """at_tune picks a launch shape within its search space; the solver still
    matches the oracle afterwards."""
    from paper_1911_05769_gb300 import AT_SEEDED
    M = 256
    inst = small_ensemble(n_inst=40, seed=17, M=M, log2_n=(10.0, 13.0))
    res = gpu_ensemble_run(inst, M=M, order=2, steps=200, dtype="f64", mode=AT_SEEDED, tune=20)
    t = res["tune"]
    assert t.n_tried >= 2 and 2 <= t.stages <= 4 and t.ctas >= 1 and t.steps_per_pass == 1
    assert 0 < t.best_ms <= t.first_ms
    assert res["info"].ctas == t.ctas and res["info"].stages == t.stages
    check_against_oracle(inst, res, M=M, order=2, steps=200, mode="seeded", dtype="f64")


def test_autotuner_free_mode_shapes():
    from paper_1911_05769_gb300 import AT_FREE, EnsembleSolver
    import torch
    M = 256
    inst = small_ensemble(n_inst=30, seed=18, M=M, log2_n=(10.0, 12.5))
    s = EnsembleSolver(inst, M, 2, dtype="f32", steps_per_pass=1)
    s.set_state(torch.from_numpy(W.ensemble_field(inst)).cuda())
    t = s.tune(20, AT_FREE)
    assert 1 <= t.steps_per_pass <= max(d["L"] for d in inst) + 1
    assert s.info().steps_per_pass == t.steps_per_pass
    s.close()


# ---- multi-subdomain tiles (tile_subdomains K > 1, AT_FREE and AT_SYNC) ----

@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("K,spp,order", [(2, 0, 2), (4, 4, 2), (4, 2, 4), (2, 4, 4)])
def test_multi_subdomain_tiles_free_replays(dtype, K, spp, order):
    """A tile advances K consecutive subdomains of an instance together; the
    faces between them are at delay 0 and recorded so; every recorded delay
    pattern replays in the oracle (periodic, one- and two-subdomain and
    exact-boundary instances, tiles cut short at an instance end)."""
    from paper_1911_05769_gb300 import AT_FREE
    M = 256
    inst = small_ensemble(M=M, seed=51 + K + order, log2_n=(8.0, 11.0), periodic=(0, 2))
    inst[0]["n"] = 256
    inst[2]["n"] = 768
    for j in (0, 2):
        d = inst[j]
        x, dx = W.grid(d["n"], d["length"], d["origin"])
        d["u0"] = 0.3 + 0.2 * np.sin(x) + 0.1 * np.sin(3 * x + 1)
        d["dt"] = W.dt_rule(d["u0"], dx, d["nu"])
    steps = 160
    res = gpu_ensemble_run(inst, M=M, order=order, steps=steps, dtype=dtype, mode=AT_FREE, record=True, max_ctas=2,
                           steps_per_pass=spp, tile_subdomains=K, calls=[61, 99])
    assert res["info"].tile_subdomains == K
    rec = res["rec"]
    p0 = 0
    for d in inst:
        Pj = d["n"] // M
        r = rec[:, p0:p0 + Pj, :]
        assert r.min() >= 0 and r.max() <= d["L"]
        p0 += Pj
    check_against_oracle(inst, res, M=M, order=order, steps=steps, mode="replay", dtype=dtype, delays=rec)


@pytest.mark.parametrize("spp", [0, 4])
def test_multi_subdomain_tiles_sync_is_bitwise(spp):
    """AT_SYNC with tiles of 4 subdomains (unblocked, and blocked in passes
    of 4 levels with ghost cells) equals the one-subdomain-per-tile run bit
    for bit."""
    from paper_1911_05769_gb300 import AT_SYNC
    M = 256
    inst = small_ensemble(M=M, seed=61, log2_n=(8.0, 11.0), periodic=(1,))
    one = gpu_ensemble_run(inst, M=M, order=2, steps=120, dtype="f64", mode=AT_SYNC, max_ctas=2, steps_per_pass=spp)
    four = gpu_ensemble_run(inst, M=M, order=2, steps=120, dtype="f64", mode=AT_SYNC, max_ctas=2, steps_per_pass=spp,
                            tile_subdomains=4)
    assert np.array_equal(one["u"], four["u"])
    assert np.array_equal(one["hist"], four["hist"])


def test_multi_subdomain_tiles_across_modes():
    """Seeded steps (one subdomain per tile), then free-running steps (tiles
    of 4), then seeded again, then synchronous: the flags are brought to the
    state's level whenever the tiling changes; the recorded delays replay."""
    from paper_1911_05769_gb300 import AT_FREE, AT_SEEDED, AT_SYNC
    M = 256
    inst = small_ensemble(n_inst=12, M=M, seed=62, log2_n=(9.0, 11.5))
    calls, modes = [30, 50, 40, 20], [AT_SEEDED, AT_FREE, AT_SEEDED, AT_SYNC]
    res = gpu_ensemble_run(inst, M=M, order=2, steps=140, dtype="f64", mode=AT_FREE, record=True, max_ctas=3,
                           steps_per_pass=3, tile_subdomains=4, calls=calls, modes=modes)
    check_against_oracle(inst, res, M=M, order=2, steps=140, mode="replay", dtype="f64", delays=res["rec"])


def test_multi_subdomain_tiles_compensated():
    from paper_1911_05769_gb300 import AT_FLAG_COMPENSATED, AT_FREE
    M = 256
    inst = small_ensemble(M=M, seed=63, log2_n=(8.5, 11.0))
    res = gpu_ensemble_run(inst, M=M, order=2, steps=200, dtype="f32", mode=AT_FREE, record=True, max_ctas=2,
                           steps_per_pass=4, tile_subdomains=4, flags=AT_FLAG_COMPENSATED)
    ref = oracle_ensemble(inst, M=M, order=2, steps=200, mode="replay", delays=res["rec"])
    ph, pl = split(res["u"], res["offsets"]), split(res["lo"], res["offsets"])
    for j, (u_ref, _) in ref.items():
        assert rel_linf(ph[j] + pl[j], u_ref) <= 1e-6, j


def test_autotuner_chooses_tile_subdomains():
    """In free-running mode the tuner also tries 1, 2 and 4 subdomains per
    tile and keeps the fastest shape; the run stays replayable."""
    from paper_1911_05769_gb300 import AT_FREE
    M = 256
    inst = small_ensemble(n_inst=40, seed=64, M=M, log2_n=(10.0, 12.5))
    res = gpu_ensemble_run(inst, M=M, order=2, steps=100, dtype="f64", mode=AT_FREE, record=True, tune=10,
                           steps_per_pass=1)
    t = res["tune"]
    assert t.tile_subdomains in (1, 2, 4) and res["info"].tile_subdomains == t.tile_subdomains
    assert t.n_tried >= 3
    check_against_oracle(inst, res, M=M, order=2, steps=100, mode="replay", dtype="f64", delays=res["rec"])


@pytest.mark.parametrize("kind", ["ensemble", "single"])
def test_captured_graph_replays_continue(kind):
    """at_step captured once into a CUDA graph and replayed three times equals
    three at_step calls bit for bit (the level of the state lives on the
    device), and the level reported afterwards is 3 n."""
    import torch

    from paper_1911_05769_gb300 import AT_SEEDED, EnsembleSolver, Solver
    M, n = 256, 40
    st = torch.cuda.Stream()

    def make():
        if kind == "ensemble":
            inst = small_ensemble(M=M, seed=19)
            s = EnsembleSolver(inst, M, 2, dtype="f64", stream=st)
            u0 = W.ensemble_field(inst)
        else:
            cfg = W.config("burgers1d_n4096")
            u0 = W.initial_field(cfg)
            _, dx = W.grid(cfg["N"])
            s = Solver(cfg["N"], cfg["P"], 2, 2, cfg["nu"], W.dt_rule(u0, dx, cfg["nu"]), dtype="f64", seed=1,
                       stream=st)
        with torch.cuda.stream(st):
            s.set_state(torch.from_numpy(u0).cuda())
        return s

    a = make()
    with torch.cuda.stream(st):
        for _ in range(3):
            a.step(n, AT_SEEDED)
        ua = a.state()
    b = make()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        b.step(n, AT_SEEDED)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        ub = b.state()
    assert b.info().step == 3 * n
    assert torch.equal(ua, ub)
    a.close()
    b.close()


def test_full_ensemble_fp64_sampled_instances():
    """The 2048-instance ensemble at full size (N = 3.1e7 points, P = 121001
    subdomains of 256 points, L_j in {1, 2, 3}), FP64, seeded delays, 5000
    steps, in the launch shape the benchmark uses; sampled instances (the three
    smallest, the largest and four others) against the oracle."""
    inst = W.ensemble()
    steps = 5000
    res = gpu_ensemble_run(inst, M=256, order=2, steps=steps, dtype="f64")
    n = np.array([d["n"] for d in inst])
    order = np.argsort(n)
    rng = np.random.default_rng(3)
    which = set(order[:3].tolist()) | {int(order[-1])} | set(rng.choice(np.where(n <= 8192)[0], 4).tolist())
    check_against_oracle(inst, res, M=256, order=2, steps=steps, mode="seeded", dtype="f64", which=which)


# The 2048-instance workload in FP32 state over all of its 5000 steps.  Plain
# FP32: rounding the stored field at every update, with increments that stay
# alike from step to step while the slow travelling wave crosses a point, so
# the rounding errors add up nearly linearly (up to 2.0e-3 of max|u| on the
# sampled instances, the small ones with the largest dt; the oracle's FP64
# run shows no such drift).  Bound: twice that.  The compensated state
# (hi + lo words, word-by-word stencil differences, two-sum updates) stays
# within the FP32 bar of 1e-5 over all 5000 steps.
PLAIN_FP32_BOUND_5000 = 4e-3


def _full_ensemble_sample(inst):
    n = np.array([d["n"] for d in inst])
    order = np.argsort(n)
    rng = np.random.default_rng(4)
    return set(order[:4].tolist()) | {int(order[-1])} | set(rng.choice(np.where(n <= 4096)[0], 3).tolist())


def test_full_ensemble_fp32_all_steps():
    from paper_1911_05769_gb300 import AT_FLAG_COMPENSATED
    inst = W.ensemble()
    steps = 5000
    which = _full_ensemble_sample(inst)
    ref = oracle_ensemble(inst, M=256, order=2, steps=steps, mode="seeded", which=which)
    plain = gpu_ensemble_run(inst, M=256, order=2, steps=steps, dtype="f32")
    comp = gpu_ensemble_run(inst, M=256, order=2, steps=steps, dtype="f32", flags=AT_FLAG_COMPENSATED)
    pp, ph, pl = split(plain["u"], plain["offsets"]), split(comp["u"], comp["offsets"]), split(comp["lo"], comp["offsets"])
    worst_plain = worst_comp = 0.0
    for j, (u_ref, _) in ref.items():
        worst_plain = max(worst_plain, rel_linf(pp[j], u_ref))
        e_hi = rel_linf(ph[j], u_ref)
        e_pair = rel_linf(ph[j] + pl[j], u_ref)
        assert e_hi <= TOL["f32"], (j, inst[j]["n"], e_hi)
        assert e_pair <= TOL["f32"], (j, inst[j]["n"], e_pair)
        worst_comp = max(worst_comp, e_hi)
    assert worst_plain <= PLAIN_FP32_BOUND_5000, worst_plain
    assert np.array_equal(plain["hist"], comp["hist"])


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("mode", ["seeded", "sync", "free_blocked"])
def test_compensated_ensemble_matches_oracle(mode, order):
    """Compensated FP32 state in an ensemble (periodic and exact-boundary
    instances): seeded, synchronous and blocked free-running delays (recorded,
    replayed by the oracle); the public hi words within the FP32 bar, the
    carried value hi + lo within 1e-6 (only the FP32 rounding of each
    increment and of the initial field remain)."""
    from paper_1911_05769_gb300 import AT_FLAG_COMPENSATED, AT_FREE, AT_SEEDED, AT_SYNC
    M = 256
    inst = small_ensemble(M=M, seed=31 + order, periodic=(1,))
    steps = 400
    m = {"seeded": AT_SEEDED, "sync": AT_SYNC, "free_blocked": AT_FREE}[mode]
    res = gpu_ensemble_run(inst, M=M, order=order, steps=steps, dtype="f32", mode=m, max_ctas=2,
                           record=(mode == "free_blocked"), steps_per_pass=(4 if mode == "free_blocked" else 0),
                           flags=AT_FLAG_COMPENSATED)
    omode = {"seeded": "seeded", "sync": "sync", "free_blocked": "replay"}[mode]
    ref = oracle_ensemble(inst, M=M, order=order, steps=steps, mode=omode, delays=res.get("rec"))
    ph, pl = split(res["u"], res["offsets"]), split(res["lo"], res["offsets"])
    for j, (u_ref, _) in ref.items():
        assert rel_linf(ph[j], u_ref) <= TOL["f32"], j
        assert rel_linf(ph[j] + pl[j], u_ref) <= 1e-6, (j, rel_linf(ph[j] + pl[j], u_ref))


@pytest.mark.parametrize("K", [1, 4])
def test_full_ensemble_free_blocked_replay_sampled(K):
    from paper_1911_05769_gb300 import AT_FREE
    inst = W.ensemble()
    steps = 200
    res = gpu_ensemble_run(inst, M=256, order=2, steps=steps, dtype="f64", mode=AT_FREE, record=True,
                           steps_per_pass=4, tile_subdomains=K)
    n = np.array([d["n"] for d in inst])
    which = set(np.argsort(n)[:3].tolist()) | {int(np.argmax(n))}
    check_against_oracle(inst, res, M=256, order=2, steps=steps, mode="replay", dtype="f64", delays=res["rec"],
                         which=which)
    # travelling-wave instances stay close to the exact solution
    parts = split(res["u"], res["offsets"])
    for j in which:
        d = inst[j]
        exact = W.tanh_wave(d, steps * d["dt"])
        assert np.max(np.abs(parts[j] - exact)) < 0.05 * max(d["tanh_a"], 1e-3) + 1e-3


@pytest.mark.parametrize("kind", ["single", "ensemble"])
def test_tuning_across_partitions_continues_exactly(kind):
    """at_tune times shapes with different CTA counts, so the subdomains are
    split among processing elements differently from one launch to the next
    (some faces between two PEs were inside one PE before).  With seeded delays
    the state after tuning and further steps must still equal the oracle's
    uninterrupted run of the same number of levels; free-running tuning must
    finish without a timed-out wait."""
    import torch

    from paper_1911_05769_gb300 import AT_FREE, AT_SEEDED, EnsembleSolver, Solver
    if kind == "single":
        N, P, order, L, nu = 81920, 1280, 2, 2, 0.02       # 1280 subdomains: 152, 304, 320 CTAs differ
        x, dx = W.grid(N)
        u0 = np.sin(x) + 0.5 * np.sin(3 * x + 1)
        dt = W.dt_rule(u0, dx, nu)
        mk = lambda: Solver(N, P, order, L, nu, dt, dtype="f64", seed=7)
    else:
        inst = small_ensemble(n_inst=80, seed=21, log2_n=(11.0, 12.3))
        assert sum(d["n"] for d in inst) // 256 > 4 * 152       # 152 CTAs and all co-resident differ
        u0 = W.ensemble_field(inst)
        mk = lambda: EnsembleSolver(inst, 256, 2, dtype="f64")
    s = mk()
    s.set_state(torch.from_numpy(u0).cuda())
    t = s.tune(10, AT_SEEDED)
    assert t.n_tried >= 3
    s.step(30, AT_SEEDED)
    total = s.info().step
    assert total == 30 + 3 * 10 * t.n_tried
    got = s.state().cpu().numpy()
    s.close()
    if kind == "single":
        ref, _ = oracle.run(u0, P=P, order=order, L=L, nu=nu, dt=dt, n_steps=total, delay_mode=oracle.SEEDED,
                            seed=7)
        assert rel_linf(got, ref) <= TOL["f64"]
    else:
        res = {"u": got, "offsets": list(np.concatenate([[0], np.cumsum([d["n"] for d in inst])]))}
        check_against_oracle(inst, res, M=256, order=2, steps=total, mode="seeded", dtype="f64",
                             which=set(range(0, 80, 9)))
    f = mk()
    f.set_state(torch.from_numpy(u0).cuda())
    f.tune(10, AT_FREE)
    f.step(20, AT_FREE)
    assert np.isfinite(f.state().cpu().numpy()).all()      # state() raises on a timed-out wait
    f.close()
