"""Batched execution on the GPU: each controller stepped inside the batch
gives, bit for bit, what it gives alone through the context API with the
same launch shape; graph replay equals eager launches; admission by memory;
and batch results agree with the CPU oracle."""
import numpy as np
import pytest

from cost_checks import cost_errors
from paper_2504_06437_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06437_gb300 import binding
    binding.build()
    binding.load()
    return binding


def mix(n, seed=0, K_hi=3000):
    g = W.rng(seed)
    return [W._mixed_world(g, i, seed, 64, K_hi, 10, 40, 0 if i == 3 else 5, 80) for i in range(n)]


def test_batch_equals_alone_bitwise(gpu):
    worlds = mix(6)
    with gpu.Batch(16, 256 << 20) as b:
        slots = [b.add(w.params, w.obstacles) for w in worlds]
        shapes = [b.slot_info(s) for s in slots]
        for step in range(2):
            x0s = [w.x_start for w in worlds]
            xrefs = [w.reference(w.x_start) for w in worlds]
            b.step(slots, x0s, xrefs)
            u_b = b.controls()
            st_b = [b.state(s) for s in slots]
            if step == 0:
                alone = []
                for w, sh in zip(worlds, shapes):
                    g = gpu.Controller(w.params, tiling=dict(samples_per_cta=sh["samples_per_cta"],
                                                             threads=256,
                                                             positions_per_thread=sh["positions_per_thread"]))
                    g.set_obstacles(w.obstacles)
                    alone.append(g)
            for i, (w, g) in enumerate(zip(worlds, alone)):
                g.step(w.x_start, w.reference(w.x_start))
                u0, U = g.get_control(want_U=True)
                d = g.get_debug()
                np.testing.assert_array_equal(u_b[i], u0)
                np.testing.assert_array_equal(st_b[i]["U"], U)
                np.testing.assert_array_equal(st_b[i]["costs"], d["costs"])
                assert st_b[i]["S_e"] == d["S_e_next"]
        for g in alone:
            g.close()


def test_graph_replay_equals_eager(gpu):
    worlds = mix(5, seed=2)
    outs = []
    for use_graph in (True, False):
        with gpu.Batch(8, 256 << 20) as b:
            b.set_graph(use_graph)
            slots = [b.add(w.params, w.obstacles) for w in worlds]
            us = []
            for _ in range(3):
                b.step(slots, [w.x_start for w in worlds], [w.reference(w.x_start) for w in worlds])
                us.append(b.controls())
            outs.append(np.array(us))
    np.testing.assert_array_equal(outs[0], outs[1])


def test_subsets_and_order(gpu):
    """Stepping a subset, in another order, leaves the others untouched and
    gives the same per-controller results."""
    worlds = mix(4, seed=3)
    with gpu.Batch(8, 256 << 20) as b, gpu.Batch(8, 256 << 20) as c:
        sb = [b.add(w.params, w.obstacles) for w in worlds]
        sc = [c.add(w.params, w.obstacles) for w in worlds]
        b.step(sb, [w.x_start for w in worlds], [w.reference(w.x_start) for w in worlds])
        ub = b.controls()
        order = [2, 0, 3]
        c.step([sc[i] for i in order], [worlds[i].x_start for i in order],
               [worlds[i].reference(worlds[i].x_start) for i in order])
        uc = c.controls()
        for j, i in enumerate(order):
            np.testing.assert_array_equal(uc[j], ub[i])
        assert c.state(sc[1])["iter"] == 0


def test_admission_by_memory(gpu):
    w = W.quad2d(0, K=8192, T=60)
    with gpu.Batch(64, 4 << 20) as b:
        slots = []
        with pytest.raises(gpu.MppiError) as e:
            for _ in range(64):
                slots.append(b.add(w.params, w.obstacles))
        assert e.value.code == gpu.MPPI_ENOMEM
        assert len(slots) >= 1
        free_before = b.slot_info()["pool_free"]
        b.remove(slots[0])
        assert b.slot_info()["pool_free"] > free_before
        slots[0] = b.add(w.params, w.obstacles)          # fits again
        b.step(slots, [w.x_start] * len(slots))
        assert np.all(np.isfinite(b.controls()))


def test_batch_matches_oracle(gpu, orc):
    """One batched step of all four models and a smoothed controller (window
    9, order 3) against the oracle, from the same inputs: per-sample costs,
    u*_0 and the shifted sequence of every slot."""
    worlds = [W.unicycle_small(1), W.quad2d(1, K=700, T=30), W.ackermann(1), W.quad5(1),
              W.quad2d(2, K=500, T=24)]
    worlds[-1].params.update(sgf_window=9, sgf_order=3)
    with gpu.Batch(len(worlds), 256 << 20) as b:
        slots = [b.add(w.params, w.obstacles) for w in worlds]
        ctls = [orc.new_controller(w.params) for w in worlds]
        xrefs = [w.reference(w.x_start) for w in worlds]
        b.step(slots, [w.x_start for w in worlds], xrefs)
        u = b.controls()
        for i, (w, s) in enumerate(zip(worlds, slots)):
            ro = orc.step(w.params, w.obstacles, w.x_start, xrefs[i], ctls[i])
            st = b.state(s)
            rel_max, _, ratio, _ = cost_errors(ro, st["costs"])
            assert ratio <= 1.0, (i, rel_max, ratio)
            np.testing.assert_allclose(u[i], ro["u0"], rtol=0, atol=1e-5, err_msg=str(i))
            np.testing.assert_allclose(st["U"], ro["U_next"], rtol=0, atol=1e-5, err_msg=str(i))


def test_batch_autotuned_policy_shapes_and_equals_alone(gpu):
    """mppi_batch_autotune picks a per-model policy from timed batched steps;
    a batch under that policy gives each new controller the policy's shape
    (samples per CTA capped at K), and its results still equal the
    one-controller launch of the same shape bit for bit."""
    worlds = mix(4)
    pol, ms = gpu.batch_autotune([w.params for w in worlds], [w.obstacles for w in worlds],
                                 iters=2, pool_bytes=256 << 20)
    assert ms > 0.0
    for m in range(2):
        assert pol["samples_per_cta"][m] in (8, 16, 32)
        assert pol["positions_per_thread"][m] in (0, 8, 14)
    with gpu.Batch(8, 256 << 20) as b:
        with pytest.raises(gpu.MppiError):
            b.set_policy(dict(samples_per_cta=[0, 32], positions_per_thread=[0, 0]))
        with pytest.raises(gpu.MppiError):
            b.set_policy(dict(samples_per_cta=[32, 32], positions_per_thread=[9, 0]))
        b.set_policy(pol)
        assert b.get_policy() == pol
        slots = [b.add(w.params, w.obstacles) for w in worlds]
        for w, s in zip(worlds, slots):
            sh = b.slot_info(s)
            m = int(w.params["model"])
            assert sh["samples_per_cta"] == min(pol["samples_per_cta"][m], int(w.params["K"]))
            if pol["positions_per_thread"][m]:
                assert sh["positions_per_thread"] == pol["positions_per_thread"][m]
        b.step(slots, [w.x_start for w in worlds], [w.reference(w.x_start) for w in worlds])
        u_b = b.controls()
        for i, (w, s) in enumerate(zip(worlds, slots)):
            sh = b.slot_info(s)
            with gpu.Controller(w.params, tiling=dict(samples_per_cta=sh["samples_per_cta"], threads=256,
                                                      positions_per_thread=sh["positions_per_thread"])) as g:
                g.set_obstacles(w.obstacles)
                g.step(w.x_start, w.reference(w.x_start))
                np.testing.assert_array_equal(u_b[i], g.get_control())


@pytest.mark.parametrize("model,npos", [("unicycle", 8), ("unicycle", 14), ("quad", 8), ("quad", 14),
                                        ("ackermann", 8), ("ackermann", 14), ("quad5", 8)])
def test_register_forms_equal_bitwise(gpu, model, npos):
    """A controller whose grid spans several waves runs the 80-register form
    of the step kernel; a one-wave controller the 96-register form.  The
    80-register controller gives, bit for bit, what the batch kernel gives
    for it at the same launch shape (and the batch kernel equals the
    96-register form in the test above).  All four models, 8 and 14 points
    per barrier thread."""
    if model == "unicycle":
        w = W.unicycle_stress(3, K=16384, T=40)
        small = W.unicycle_stress(3, K=512, T=40)
    elif model == "quad":
        w = W.quad2d(3, K=16384, T=30)
        small = W.quad2d(3, K=512, T=30)
    else:
        w = W.PRESETS[model](3, K=16384, T=30)
        small = W.PRESETS[model](3, K=512, T=30)
    shape = dict(samples_per_cta=20, threads=256, positions_per_thread=npos)
    with gpu.Controller(small.params, tiling=shape) as g:
        g.set_obstacles(small.obstacles)
        assert g.kernel_regs() == 96
    with gpu.Batch(4, 256 << 20) as b, gpu.Controller(w.params, tiling=shape) as g:
        g.set_obstacles(w.obstacles)
        assert g.tiling()["n_ctas"] == (16384 + 19) // 20
        assert g.kernel_regs() == 80
        slot = b.add(w.params, w.obstacles, tiling=shape)
        for _ in range(2):
            xr = w.reference(w.x_start)
            b.step([slot], [w.x_start], [xr])
            u_b = b.controls()
            st = b.state(slot)
            g.step(w.x_start, xr)
            u0, U = g.get_control(want_U=True)
            d = g.get_debug()
            np.testing.assert_array_equal(u_b[0], u0)
            np.testing.assert_array_equal(st["U"], U)
            np.testing.assert_array_equal(st["costs"], d["costs"])


def test_batch_all_four_models_equal_alone(gpu):
    """One batched launch holding all four models (unicycle, 6-state
    quadrotor, Ackermann vehicle, 5-state quadrotor): each controller's
    result equals, bit for bit, its step alone at the same launch shape."""
    worlds = [W.unicycle_small(1), W.quad2d(1, K=1024, T=20), W.ackermann(1), W.quad5(1)]
    with gpu.Batch(8, 256 << 20) as b:
        slots = [b.add(w.params, w.obstacles) for w in worlds]
        shapes = [b.slot_info(s) for s in slots]
        b.step(slots, [w.x_start for w in worlds], [w.reference(w.x_start) for w in worlds])
        u_b = b.controls()
        st_b = [b.state(s) for s in slots]
    for i, (w, sh) in enumerate(zip(worlds, shapes)):
        with gpu.Controller(w.params, tiling=dict(samples_per_cta=sh["samples_per_cta"], threads=256,
                                                  positions_per_thread=sh["positions_per_thread"])) as g:
            g.set_obstacles(w.obstacles)
            g.step(w.x_start, w.reference(w.x_start))
            u0, U = g.get_control(want_U=True)
            d = g.get_debug()
        np.testing.assert_array_equal(u_b[i], u0)
        np.testing.assert_array_equal(st_b[i]["U"], U)
        np.testing.assert_array_equal(st_b[i]["costs"], d["costs"])


def test_batch_with_smoothing_equals_alone(gpu):
    """Slots with and without Savitzky-Golay smoothing of the update in one
    batched launch, each equal bit for bit to its step alone."""
    worlds = [W.unicycle_small(2), W.quad2d(2, K=1024, T=20), W.ackermann(2), W.quad5(2)]
    sgf = [(5, 2), (0, 0), (9, 3), (3, 1)]
    params = [dict(w.params, sgf_window=a, sgf_order=o) for w, (a, o) in zip(worlds, sgf)]
    with gpu.Batch(8, 256 << 20) as b:
        slots = [b.add(p, w.obstacles) for p, w in zip(params, worlds)]
        shapes = [b.slot_info(s) for s in slots]
        for _ in range(2):
            b.step(slots, [w.x_start for w in worlds], [w.reference(w.x_start) for w in worlds])
        u_b = b.controls()
        st_b = [b.state(s) for s in slots]
    for i, (w, p, sh) in enumerate(zip(worlds, params, shapes)):
        with gpu.Controller(p, tiling=dict(samples_per_cta=sh["samples_per_cta"], threads=256,
                                           positions_per_thread=sh["positions_per_thread"])) as g:
            g.set_obstacles(w.obstacles)
            for _ in range(2):
                g.step(w.x_start, w.reference(w.x_start))
            u0, U = g.get_control(want_U=True)
        np.testing.assert_array_equal(u_b[i], u0)
        np.testing.assert_array_equal(st_b[i]["U"], U)
