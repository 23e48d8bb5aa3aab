"""GPU parity: the CUDA step (through the C ABI) against the CPU FP64 oracle,
element by element, on the same seeded inputs.

Tolerances: per-sample cost-to-go within 1e-4 relative (relative to
max(|S|, 1)), widened for samples that pass close to an obstacle by what
the FP32 rollout's positions allow (cost_checks), the updated control
sequence U* within 1e-5 absolute, the set
of collided samples identical wherever the oracle's min h is farther than
H_MARGIN from zero (closer samples are reported, not asserted).  Philox words
are compared bit for bit."""
import dataclasses
import json
import math

import numpy as np
import pytest

from paper_2504_06437_gb300 import workloads as W
from cost_checks import COST_RTOL, cost_errors
from weight_checks import check_weights

pytestmark = pytest.mark.gpu

U_ATOL = 1e-5
H_MARGIN = 1e-4


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06437_gb300 import binding
    binding.build()
    binding.load()
    return binding


def compare_step(ro, dbg, u0, U_next, label="", lam=1.0):
    rel_max, beyond, ratio, k = cost_errors(ro, dbg["costs"])
    assert ratio <= 1.0, (f"{label} cost error {ratio:.3f} of its tolerance at k={k} "
                          f"(largest relative error {rel_max:.3e}, {beyond} beyond {COST_RTOL})")
    sure = np.abs(ro["minh"]) > H_MARGIN
    mism = np.nonzero((ro["coll"] != dbg["coll"]) & sure)[0]
    assert mism.size == 0, f"{label} collided set differs at {mism[:10]}"
    np.testing.assert_allclose(dbg["Ustar"], ro["Ustar"], rtol=0, atol=U_ATOL, err_msg=label)
    np.testing.assert_allclose(u0, ro["u0"], rtol=0, atol=U_ATOL, err_msg=label)
    np.testing.assert_allclose(U_next, ro["U_next"], rtol=0, atol=U_ATOL, err_msg=label)
    assert abs(dbg["weights"].sum() - 1.0) < 1e-6
    check_weights(ro, dbg, lam, label)
    assert dbg["beta_used"] == pytest.approx(ro["beta_used"], rel=1e-5, abs=1e-6)
    assert dbg["beta_d"] == pytest.approx(ro["beta_d"], rel=1e-5, abs=1e-6)
    assert dbg["CB_star"] == pytest.approx(ro["CB_star"], rel=1e-4, abs=1e-4)
    assert dbg["S_e_next"] == pytest.approx(ro["S_e_next"], rel=1e-5)
    return dict(cost_rel=rel_max, cost_beyond_rtol=beyond, cost_tol_ratio=ratio,
                U_abs=float(np.abs(dbg["Ustar"] - ro["Ustar"]).max()),
                w_abs=float(np.abs(dbg["weights"] - ro["weights"]).max()))


def run_pair(gpu, orc, world, steps=1, tiling=None, u_init=None):
    """Run the oracle and the GPU side by side for `steps` receding-horizon
    iterations.  The plant is advanced with the oracle's u0, and before each
    step the GPU controller is given the oracle's controller state (U, S_e,
    beta, iteration), so every step is compared from identical inputs: the
    tolerances are per step, and the exponentiated weights would otherwise
    amplify the previous step's admissible differences."""
    p = world.params
    ctl = orc.new_controller(p, u_init)
    errs = []
    with gpu.Controller(p, u_init=u_init, tiling=tiling) as g:
        g.set_obstacles(world.obstacles)
        if p.get("grid") is not None:
            g.set_grid(p["grid"], p["grid_ox"], p["grid_oy"], p["grid_res"])
        x = world.x_start.copy()
        for i in range(steps):
            if i > 0:
                g.set_state(ctl.U, ctl.S_e, ctl.beta, ctl.first, ctl.iter)
            xref = world.reference(x)
            ro = orc.step(p, world.obstacles, x, xref, ctl)
            g.step(x, xref)
            u0, U_next = g.get_control(want_U=True)
            dbg = g.get_debug()
            errs.append(compare_step(ro, dbg, u0, U_next, label=f"{world.name} step {i}",
                                     lam=float(p["lambda"])))
            x = orc.dynamics(p, x, ro["u0"])
    return errs


def test_closed_loop_free_running(gpu, orc):
    """Both controllers run on their own for 20 steps, each driving its own
    FP64 plant: a behavioural check (no resynchronisation).  Per-step
    differences within the parity tolerances are amplified by the weights of
    later steps (the controller is a stochastic optimiser), so the bound is
    on the executed trajectory: within 5 cm after 20 steps."""
    w = W.unicycle_small(0)
    p = w.params
    ctl = orc.new_controller(p)
    xo = w.x_start.copy()
    xg = w.x_start.copy()
    with gpu.Controller(p) as g:
        g.set_obstacles(w.obstacles)
        for _ in range(20):
            ro = orc.step(p, w.obstacles, xo, w.reference(xo), ctl)
            g.step(xg, w.reference(xg))
            ug = g.get_control()
            xo = orc.dynamics(p, xo, ro["u0"])
            xg = orc.dynamics(p, xg, ug)
    assert np.abs(xo - xg).max() < 5e-2, (xo, xg)


def test_philox_words_bit_exact(gpu, orc):
    p = W.base_params(W.UNICYCLE, K=8, T=4, dt=0.05, seed=0x123456789ABCDEF)
    raw, _ = gpu.debug_draws(p, 0.4, (7 << 32) + 3, 37, 11)
    it = (7 << 32) + 3
    key = [p["seed"] & 0xFFFFFFFF, p["seed"] >> 32]
    for k in range(37):
        for t in range(11):
            ref = orc.philox4x32_10([k, t, it & 0xFFFFFFFF, it >> 32], key)
            np.testing.assert_array_equal(raw[k, t], ref)


@pytest.mark.parametrize("sig", [[0.5, 0.0, 0.0, 0.5], [0.5, 0.2, 0.2, 0.3]])
def test_nln_draws_match_oracle(gpu, orc, sig):
    p = W.base_params(W.UNICYCLE, K=8, T=4, dt=0.05, seed=11)
    p["sigma"] = sig
    _, du = gpu.debug_draws(p, 0.7, 5, 64, 30)
    ref, _ = orc.noise_batch(p, 0.7, 64, 30, 5)
    np.testing.assert_allclose(du, ref, rtol=2e-6, atol=2e-6)


def test_unicycle_small_closed_loop(gpu, orc):
    """Config 1 (K=256, T=30, 10 obstacles), five receding-horizon steps."""
    run_pair(gpu, orc, W.unicycle_small(0), steps=5)


def test_quad_ragged_tiles(gpu, orc):
    """Planar quadrotor, K=1000 (ragged last tile), T=50, 40 obstacles, 7 shape points."""
    w = W.quad2d(1, K=1000, T=50)
    run_pair(gpu, orc, w, steps=3)


@pytest.mark.parametrize("tiling", [
    dict(samples_per_cta=32, threads=64, positions_per_thread=8, chunk_steps=0),
    dict(samples_per_cta=7, threads=512, positions_per_thread=14, chunk_steps=3),
    dict(samples_per_cta=1, threads=128, positions_per_thread=14, chunk_steps=0),
    dict(samples_per_cta=20, threads=256, positions_per_thread=8, chunk_steps=11),
])
def test_tilings_agree_with_oracle(gpu, orc, tiling):
    w = W.quad2d(2, K=777, T=23)
    run_pair(gpu, orc, w, steps=2, tiling=tiling)
    w = W.unicycle_small(2)
    w.params.update(K=999, T=41)
    run_pair(gpu, orc, w, steps=2, tiling=tiling)


def test_no_obstacles(gpu, orc):
    w = W.unicycle_small(3)
    w.obstacles = np.zeros((0, 3))
    errs = run_pair(gpu, orc, w, steps=2)
    assert errs


def test_single_sample_single_step(gpu, orc):
    w = W.unicycle_small(4)
    w.params.update(K=1, T=1)
    run_pair(gpu, orc, w, steps=3)


def test_many_collisions(gpu, orc):
    """Obstacles placed on the straight path: many samples collide."""
    w = W.unicycle_small(5)
    line = np.linspace(1.3, 2.5, 6)
    w.obstacles = np.array([[x + 0.12, x - 0.12, 0.1] for x in line])
    w.params.update(K=2048)
    p = w.params
    ctl = orc.new_controller(p, np.tile([1.5, 0.0], (p["T"], 1)))
    with gpu.Controller(p, u_init=np.tile([1.5, 0.0], (p["T"], 1))) as g:
        g.set_obstacles(w.obstacles)
        x = w.x_start
        xref = w.reference(x)
        ro = orc.step(p, w.obstacles, x, xref, ctl)
        g.step(x, xref)
        u0, Un = g.get_control(want_U=True)
        compare_step(ro, g.get_debug(), u0, Un, "collisions")
    assert 0 < ro["coll"].sum() < p["K"]


def test_max_sizes(gpu, orc):
    """T = 256 (limit), 4096 obstacles (limit), 8 shape points."""
    w = W.unicycle_small(6)
    g = W.rng(6)
    w.obstacles = W.obstacle_field(g, 4096, (-40, -40), (50, 50), 0.05, 0.3,
                                   keep_clear=(w.x_start, w.goal))
    w.params.update(K=96, T=256, shape=np.array([[0.2 * math.cos(a), 0.2 * math.sin(a)]
                                                  for a in np.linspace(0, 2 * math.pi, 8, endpoint=False)]))
    run_pair(gpu, orc, w, steps=1)


def bench_tiling(gpu, w):
    """The launch shape bench.py times for this workload: the autotuner's
    pick, made the same way (10 timed steps per candidate at least, each
    alone after a 256 MB write, as the bench times them)."""
    tiling, _ = gpu.autotune(w.params, w.obstacles, iters=10, flush_bytes=256 << 20)
    return tiling


def test_quad_full_size_bench_config(gpu, orc):
    """The benchmark workload (K=4096, T=50, 40 obstacles, 7 shape points) in
    the launch shape the benchmark uses (the autotuner's pick) and in the
    library's default shape, all samples compared."""
    w = W.quad2d(0)
    run_pair(gpu, orc, w, steps=2, tiling=bench_tiling(gpu, w))
    run_pair(gpu, orc, w, steps=1)


@pytest.mark.parametrize("world", ["unicycle_stress", "quad2d_corridor"])
def test_full_size_three_steps_with_collisions(gpu, orc, world):
    """Full-size colliding worlds for three receding-horizon steps in the
    launch shape bench.py times: the stress workload (K 65536, T 100, 200
    circles) from a nominal sequence that grazes the circle ahead of the
    start, and the quadrotor (K 4096, T 50, 7 shape points) with six circles
    on its flight line; thousands of samples collide.  Every sample's cost,
    the collided set, U*, the shifted sequence, C_B, S_e and the plant's
    barrier state carried into the next step, against the oracle at each
    step.  Some samples pass within h = 1e-3 of a circle without touching
    it; their costs are held to the position-error term of the tolerance
    (cost_checks), which there is what the FP32 rollout's positions allow."""
    w = W.PRESETS[world](0)
    u_init = None
    if world == "unicycle_stress":
        u_init = np.tile(np.array([1.0, 0.5]), (int(w.params["T"]), 1))
    errs = run_pair(gpu, orc, w, steps=3, tiling=bench_tiling(gpu, w), u_init=u_init)
    print("THREE_STEPS " + world + " " + json.dumps(errs))


@pytest.mark.parametrize("shape", ["bench", "default"])
def test_stress_config_sampled(gpu, orc, shape):
    """K=65536, T=100, 200 obstacles: many tile groups.  Costs of 512 sampled
    samples against the oracle; weights sum to one; U* within the box.  Run
    in the launch shape bench.py times (the autotuner's pick, which takes
    the 80-register form of the kernel on GB300) and in the default shape."""
    w = W.unicycle_stress(0)
    p = w.params
    ctl = orc.new_controller(p)
    tiling = bench_tiling(gpu, w) if shape == "bench" else None
    with gpu.Controller(p, tiling=tiling) as g:
        g.set_obstacles(w.obstacles)
        x = w.x_start
        xref = w.reference(x)
        g.step(x, xref)
        g.get_control()
        dbg = g.get_debug()
    ks = np.unique(np.concatenate([np.arange(0, p["K"], 131), [p["K"] - 1],
                                   np.argsort(dbg["costs"])[:32]]))
    ro = orc.sample_costs(p, w.obstacles, x, xref, ctl, ks)
    assert cost_errors(ro, dbg["costs"][ks])[2] <= 1.0
    sure = np.abs(ro["minh"]) > H_MARGIN
    assert np.all((ro["coll"] == dbg["coll"][ks]) | ~sure)
    assert abs(dbg["weights"].sum() - 1.0) < 1e-6
    assert np.all(dbg["Ustar"] >= np.array(p["u_min"]) - 1e-12)
    assert np.all(dbg["Ustar"] <= np.array(p["u_max"]) + 1e-12)


def test_bounded_device_wait_expires_and_device_stays_usable(gpu, orc):
    """The wait that guards the obstacle staging is bounded: on a barrier that
    nothing completes it gives up after its cycle limit (about 1 ms here) and
    the host sees MPPI_ETIMEOUT; the device then runs a normal step that
    matches the oracle.  No fault or hang is involved."""
    lib = gpu.load()
    assert lib.mppi_debug_wait_probe(2_000_000, 1) == gpu.MPPI_OK
    assert lib.mppi_debug_wait_probe(2_000_000, 0) == gpu.MPPI_ETIMEOUT
    assert b"expired" in lib.mppi_last_error()
    assert lib.mppi_debug_wait_probe(0, 0) == gpu.MPPI_EINVAL
    run_pair(gpu, orc, W.unicycle_small(3), steps=1)


def test_checkpoint_resume_bit_exact(gpu, orc):
    w = W.quad2d(7, K=512, T=30)
    p = w.params
    x = w.x_start
    xref = w.reference(x)
    with gpu.Controller(p) as a, gpu.Controller(p) as b:
        a.set_obstacles(w.obstacles)
        b.set_obstacles(w.obstacles)
        a.step(x, xref)
        a.get_control()
        st = a.get_state()
        b.set_state(st["U"], st["S_e"], st["beta"], st["first"], st["iter"])
        a.step(x, xref)
        ua = a.get_control()
        b.step(x, xref)
        ub = b.get_control()
        np.testing.assert_array_equal(ua, ub)
        np.testing.assert_array_equal(a.get_debug()["costs"], b.get_debug()["costs"])


def test_repeatable(gpu, orc):
    w = W.quad2d(8, K=2000, T=40)
    outs = []
    for _ in range(2):
        with gpu.Controller(w.params) as g:
            g.set_obstacles(w.obstacles)
            g.step(w.x_start, w.reference(w.x_start))
            outs.append((g.get_control(), g.get_debug()["costs"]))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_error_paths(gpu):
    w = W.unicycle_small(0)
    with gpu.Controller(w.params) as g:
        with pytest.raises(gpu.MppiError) as e:
            g.get_control()
        assert e.value.code == gpu.MPPI_ESTATE
        bad = w.obstacles.copy()
        bad[0, 2] = -1.0
        with pytest.raises(gpu.MppiError) as e:
            g.set_obstacles(bad)
        assert e.value.code == gpu.MPPI_EINVAL
        bad[0] = [np.nan, 0, 1]
        with pytest.raises(gpu.MppiError):
            g.set_obstacles(bad)
        with pytest.raises(gpu.MppiError):
            g.set_obstacles(np.zeros((5000, 3)))
        with pytest.raises(gpu.MppiError):
            g.step([np.nan, 0, 0])
        g.set_obstacles(w.obstacles)
        g.step(w.x_start)          # xref NULL -> goal repeated
        u0 = g.get_control()
        assert np.all(np.isfinite(u0))


def test_back_to_back_steps_without_sync(gpu):
    """mppi_step stages its inputs in two mapped host buffers used in turn;
    the kernel reads them over the host link.  Five steps enqueued without a
    synchronisation, each from a different measured state, give bit for bit
    what the same steps give with a synchronisation after each: a staging
    buffer is never rewritten while a kernel still reads it."""
    w = W.quad2d(2)
    xs = [w.x_start + 0.05 * i * np.array([1.0, -0.5, 0.0, 0.1, 0.0, 0.02]) for i in range(5)]
    refs = [w.reference(x) for x in xs]
    with gpu.Controller(w.params) as a, gpu.Controller(w.params) as b:
        a.set_obstacles(w.obstacles)
        b.set_obstacles(w.obstacles)
        for x, r in zip(xs, refs):
            a.step(x, r)
            ua, Ua = a.get_control(want_U=True)
        for x, r in zip(xs, refs):
            b.step(x, r)
        ub, Ub = b.get_control(want_U=True)
        np.testing.assert_array_equal(ua, ub)
        np.testing.assert_array_equal(Ua, Ub)


@pytest.mark.parametrize("name", ["ackermann", "quad5"])
def test_paper_models_closed_loop(gpu, orc, name):
    """The paper's own plant models (Eq. 14 vehicle with 8 shape points,
    Eq. 12 five-state quadrotor with 7) on their mission presets, three
    receding-horizon steps, every sample compared."""
    run_pair(gpu, orc, W.PRESETS[name](0), steps=3)


@pytest.mark.parametrize("name", ["ackermann", "quad5"])
def test_paper_models_ragged_and_large(gpu, orc, name):
    """Ragged tiles (K not a multiple of the tile) and a grid of several
    waves, in the launch shapes a user would get by default."""
    w = W.PRESETS[name](1, K=777, T=23)
    run_pair(gpu, orc, w, steps=1, tiling=dict(samples_per_cta=13, threads=128,
                                               positions_per_thread=8))
    run_pair(gpu, orc, W.PRESETS[name](2, K=16384, T=30), steps=1)


def _smoothed(world, window, order):
    return dataclasses.replace(world, params=dict(world.params, sgf_window=window,
                                                  sgf_order=order))


@pytest.mark.parametrize("name,window,order", [
    ("unicycle_small", 5, 2),   # T 30
    ("quad2d", 11, 3),          # T 50, 7 shape points
    ("ackermann", 7, 4),        # T 20
    ("quad5", 3, 0),            # T 20: three-step moving average
])
def test_sgf_closed_loop(gpu, orc, name, window, order):
    """Algorithm 1's SGF on the update: the step's Savitzky-Golay weights
    (built on the device from the Gram-polynomial recurrence) against the
    oracle's per-window least-squares fit, three receding-horizon steps on
    each model, every sample and every U* entry compared."""
    run_pair(gpu, orc, _smoothed(W.PRESETS[name](4), window, order), steps=3)


@pytest.mark.parametrize("T,window,order,tiling", [
    (21, 21, 2, None),                   # one window for every t
    (37, 37, 6, None),                   # the widest window T allows, highest order
    (23, 7, 6, dict(samples_per_cta=13, threads=128, positions_per_thread=8)),  # order W-1
    (40, 15, 1, dict(samples_per_cta=7, threads=512, positions_per_thread=14)),
])
def test_sgf_edges_and_ragged(gpu, orc, T, window, order, tiling):
    """Windows as wide as the horizon, the highest order, order W - 1 (the
    identity) and ragged tiles in several launch shapes."""
    w = _smoothed(W.quad2d(5, K=777, T=T), window, order)
    run_pair(gpu, orc, w, steps=1, tiling=tiling)


def test_sgf_widest_window(gpu, orc):
    """The largest window the library takes (63 steps) at T = 70."""
    run_pair(gpu, orc, _smoothed(W.quad2d(6, K=512, T=70), 63, 5), steps=2)


def test_sgf_large_grid(gpu, orc):
    """Several waves of tiles and a two-level merge with smoothing on."""
    run_pair(gpu, orc, _smoothed(W.quad2d(7, K=16384, T=50), 9, 2), steps=1)


@pytest.mark.parametrize("window,order", [(4, 1), (65, 2), (5, 5), (9, 7), (-3, 0), (31, 2)])
def test_sgf_rejects_bad_parameters(gpu, window, order):
    """Even, too wide (65 > 63, or 31 > T = 30), negative windows and orders
    >= window or > 6 are refused at creation with MPPI_EINVAL."""
    w = _smoothed(W.unicycle_small(0), window, order)
    with pytest.raises(gpu.MppiError) as e:
        gpu.Controller(w.params)
    assert e.value.code == gpu.MPPI_EINVAL


# ------------------------------------------------ grid map (Sec. V-C)

def test_grid_mission_closed_loop(gpu, orc):
    """The vehicle mission with its obstacles as a 1001 x 301 signed-distance
    grid (no circles): three receding-horizon steps, every sample's cost,
    the collided set and U* against the oracle's bilinear lookups."""
    run_pair(gpu, orc, W.ackermann_grid(0), steps=3)


@pytest.mark.parametrize("tiling", [dict(samples_per_cta=13, threads=128, positions_per_thread=8),
                                    dict(samples_per_cta=9, threads=256, positions_per_thread=14)])
def test_grid_ragged_tiles(gpu, orc, tiling):
    """Ragged last tile (K 777) and both point counts per barrier thread."""
    run_pair(gpu, orc, W.ackermann_grid(1, K=777, T=23), steps=1, tiling=tiling)


def test_grid_with_circles_and_smoothing(gpu, orc):
    """Grid map and circle obstacles together (their terms add), with the
    update smoothed, on the 6-state quadrotor: the grid form of the kernel
    carries both passes."""
    w = W.quad2d(3, K=2048, T=40)
    lo = w.obstacles[:, :2].min(axis=0) - 3.0
    g = W.sdf_grid(w.obstacles[::3], [], lo[0], lo[1], 0.05, 400, 300)
    p = dict(w.params, grid=g, grid_ox=float(lo[0]), grid_oy=float(lo[1]), grid_res=0.05,
             sgf_window=7, sgf_order=2)
    run_pair(gpu, orc, dataclasses.replace(w, params=p), steps=2)


def test_grid_collisions(gpu, orc):
    """A wall 0.2 m ahead of the vehicle's front at 0.5 m/s: about 600 of the
    1024 samples reach h <= 0 on the grid; the collided set and the
    collision costs match the oracle."""
    w = W.ackermann(2, K=1024, T=20)
    xs = w.x_start.copy()
    xs[3] = 0.5
    g = W.sdf_grid([], [(7.2, 10.0, 8.0, 20.0)], 0.0, 5.0, 0.02, 600, 600)
    p = dict(w.params, grid=g, grid_ox=0.0, grid_oy=5.0, grid_res=0.02)
    world = dataclasses.replace(w, params=p, obstacles=np.zeros((0, 3)), x_start=xs)
    ctl = orc.new_controller(p)
    xref = world.reference(world.x_start)
    ro = orc.step(p, world.obstacles, world.x_start, xref, ctl)
    assert 50 < int(ro["coll"].sum()) < 1000
    run_pair(gpu, orc, world, steps=2)


def test_grid_removed_is_plain_kernel_bit_for_bit(gpu):
    """Setting a map and removing it again leaves a controller whose steps
    equal, bit for bit, those of a controller that never had one."""
    w = W.ackermann(3)
    g = W.ackermann_grid(3).params["grid"]
    with gpu.Controller(w.params) as a, gpu.Controller(w.params) as b:
        a.set_obstacles(w.obstacles)
        b.set_obstacles(w.obstacles)
        a.set_grid(g, 0.0, 0.0, 0.1)
        a.step(w.x_start, w.reference(w.x_start))
        a.get_control()
        a.set_grid(None)
        b.step(w.x_start, w.reference(w.x_start))
        b.get_control()
        st = b.get_state()
        a.set_state(st["U"], st["S_e"], st["beta"], st["first"], st["iter"])
        for _ in range(2):
            a.step(w.x_start, w.reference(w.x_start))
            b.step(w.x_start, w.reference(w.x_start))
        ua, Ua = a.get_control(want_U=True)
        ub, Ub = b.get_control(want_U=True)
        np.testing.assert_array_equal(ua, ub)
        np.testing.assert_array_equal(Ua, Ub)
        np.testing.assert_array_equal(a.get_debug()["costs"], b.get_debug()["costs"])


def test_grid_rejects_bad_maps(gpu):
    w = W.ackermann(0)
    with gpu.Controller(w.params) as c:
        good = np.zeros((4, 5), dtype=np.float32)
        for args in [(np.zeros((1, 5)), 0.0, 0.0, 0.1), (np.zeros((4, 1)), 0.0, 0.0, 0.1),
                     (good, 0.0, 0.0, 0.0), (good, 0.0, 0.0, -1.0), (good, np.nan, 0.0, 0.1),
                     (np.full((4, 5), np.inf), 0.0, 0.0, 0.1)]:
            with pytest.raises(gpu.MppiError) as e:
                c.set_grid(*args)
            assert e.value.code == gpu.MPPI_EINVAL
        c.set_grid(good, 0.0, 0.0, 0.1)
        c.set_grid(None)


def test_grid_autotune(gpu, orc):
    """The grid-aware autotuner runs the grid form of the kernel on every
    candidate and returns a launch shape under which the step matches the
    oracle."""
    w = W.ackermann_grid(2, K=512, T=20)
    tiling, us = gpu.autotune(w.params, w.obstacles, iters=3)
    assert us > 0 and tiling["threads"] in (128, 256, 512)
    run_pair(gpu, orc, w, steps=1, tiling=tiling)
    tiling, us = gpu.autotune(w.params, w.obstacles, iters=3, flush_bytes=64 << 20)
    assert us > 0 and tiling["threads"] in (128, 256, 512)
    run_pair(gpu, orc, w, steps=1, tiling=tiling)


@pytest.mark.parametrize("name", ["unicycle_small", "quad5"])
def test_grid_other_models(gpu, orc, name):
    """The grid form on the unicycle and the 5-state quadrotor: each world's
    circles rasterised into a signed-distance grid (no circles passed), two
    receding-horizon steps against the oracle."""
    w = W.PRESETS[name](5)
    lo = w.obstacles[:, :2].min(axis=0) - 2.0
    hi = w.obstacles[:, :2].max(axis=0) + 2.0
    res = 0.05
    nx, ny = int((hi[0] - lo[0]) / res) + 2, int((hi[1] - lo[1]) / res) + 2
    g = W.sdf_grid(w.obstacles, [], lo[0], lo[1], res, nx, ny)
    p = dict(w.params, grid=g, grid_ox=float(lo[0]), grid_oy=float(lo[1]), grid_res=res)
    run_pair(gpu, orc, dataclasses.replace(w, params=p, obstacles=np.zeros((0, 3))), steps=2)


def test_control_readback_paths(gpu):
    """mppi_get_control after host-input steps (it returns once the step's
    fenced sequence word reaches the host mirror) and after device-input
    steps (no mirror: u0 copied from device memory) returns exactly the
    step's u*_0, a fresh one every step; after mppi_set_state to an earlier
    state, the same inputs give the same control again."""
    torch = pytest.importorskip("torch")
    w = W.quad2d(4, K=1024, T=30)
    xs = [w.x_start + 0.03 * i for i in range(6)]
    refs = [w.reference(x) for x in xs]
    with gpu.Controller(w.params) as g:
        g.set_obstacles(w.obstacles)
        seen, saved = [], None
        for i, (x, xr) in enumerate(zip(xs, refs)):
            if i == 3:
                saved = g.get_state()
            if i % 2 == 0:
                g.step(x, xr)
            else:
                d = torch.tensor(np.concatenate([x, xr.ravel()]), dtype=torch.float64,
                                 device="cuda")
                g.step_device(d.data_ptr(), d.data_ptr() + 8 * len(x))
            u0 = g.get_control()
            dbg = g.get_debug()
            np.testing.assert_array_equal(u0, dbg["Ustar"][0])
            assert dbg["iter"] == i + 1
            seen.append(u0.copy())
        assert len({tuple(u) for u in seen}) == len(seen)
        g.set_state(saved["U"], saved["S_e"], saved["beta"], saved["first"], saved["iter"])
        g.step(xs[3], refs[3])
        np.testing.assert_array_equal(g.get_control(), seen[3])
        g.step(xs[4], refs[4])
        np.testing.assert_array_equal(g.get_control(), seen[4])
