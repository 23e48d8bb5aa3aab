"""Continuous-batching serving runtime on the GPU: requests that arrive
while batches are in flight are served by later, overlapping batches; each
robot's result is the same, bit for bit, as the robot alone through the
context API with the same launch shape; admission by memory."""
import time

import numpy as np
import pytest

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


def wait_all(srv, n, timeout=60.0):
    got = []
    t0 = time.time()
    while len(got) < n:
        got += srv.poll()
        assert time.time() - t0 < timeout, "requests did not complete"
    return got


@pytest.mark.parametrize("mode", ["lanes", "device_queue"])
def test_served_results_equal_alone(gpu, mode):
    """Staggered arrivals over three closed-loop rounds; each robot's controls
    equal the same robot alone, bit for bit.  device_queue: the resident
    kernel takes requests that arrive while it runs."""
    g = W.rng(11)
    worlds = [W._mixed_world(g, i, 11, 256, 6000, 10, 60, 5, 120) for i in range(7)]
    rounds = 3
    with gpu.Server(16, 512 << 20, lanes=2) as srv:
        if mode == "device_queue":
            srv.set_policy(small_ops_max=2e7, device_queue=True)
        robots = [srv.join(w.params, w.obstacles) for w in worlds]
        assert all(r is not None for r in robots)
        x = {r: w.x_start.copy() for r, w in zip(robots, worlds)}
        xs = {r: [] for r in robots}
        us = {r: [] for r in robots}
        pending = set()
        # staggered arrivals: robots submit at different times, while
        # earlier batches are still on the GPU
        order = list(robots)
        done_rounds = {r: 0 for r in robots}
        for r in order:
            xs[r].append(x[r].copy())
            srv.submit(r, x[r], worlds[robots.index(r)].reference(x[r]))
            pending.add(r)
            time.sleep(0.0005)
        t0 = time.time()
        while pending:
            for (r, u0, x1, lat, st) in srv.poll():
                assert st == 0 and lat > 0
                us[r].append(u0.copy())
                pending.discard(r)
                done_rounds[r] += 1
                if done_rounds[r] < rounds:
                    w = worlds[robots.index(r)]
                    x[r] = x1[: w.n].copy()
                    xs[r].append(x[r].copy())
                    srv.submit(r, x[r], w.reference(x[r]))
                    pending.add(r)
            assert time.time() - t0 < 60
        st = srv.stats()
        assert st["requests"] == rounds * len(robots)
        assert st["batches"] < st["requests"]          # requests shared launches
    for r, w in zip(robots, worlds):
        p = w.params
        S = min(32, p["K"])
        # the slot's launch shape: samples_per_cta as admitted (32, halved to fit)
        with gpu.Batch(2, 64 << 20) as b:
            sl = b.add(p, w.obstacles)
            info = b.slot_info(sl)
        with gpu.Controller(p, tiling=dict(samples_per_cta=info["samples_per_cta"], threads=256,
                                           positions_per_thread=info["positions_per_thread"])) as c:
            c.set_obstacles(w.obstacles)
            for k in range(rounds):
                c.step(xs[r][k], w.reference(xs[r][k]))
                np.testing.assert_array_equal(c.get_control(), us[r][k])


def test_admission_refused_then_granted(gpu):
    w = W.quad2d(2, K=8192, T=60)
    with gpu.Server(64, 4 << 20, lanes=1) as srv:
        robots = []
        while True:
            r = srv.join(w.params, w.obstacles)
            if r is None:
                break
            robots.append(r)
            assert len(robots) < 64
        assert robots
        srv.submit(robots[0], w.x_start)
        wait_all(srv, 1)
        srv.leave(robots[0])
        r = srv.join(w.params, w.obstacles)
        assert r is not None
        srv.submit(r, w.x_start)
        (rid, u0, x1, lat, st), = wait_all(srv, 1)
        assert rid == r and st == 0 and np.all(np.isfinite(u0))


@pytest.mark.parametrize("mode", ["lanes", "device_queue"])
def test_many_requests_complete(gpu, mode):
    g = W.rng(5)
    worlds = [W._mixed_world(g, i, 5, 128, 2048, 10, 40, 5, 60) for i in range(40)]
    with gpu.Server(64, 512 << 20, lanes=3) as srv:
        if mode == "device_queue":
            srv.set_policy(small_ops_max=0.0, device_queue=True)
        robots = [srv.join(w.params, w.obstacles) for w in worlds]
        for r, w in zip(robots, worlds):
            srv.submit(r, w.x_start)
        got = wait_all(srv, len(robots))
        assert sorted(x[0] for x in got) == sorted(robots)
        with pytest.raises(gpu.MppiError):
            srv.submit(robots[0], worlds[0].x_start)
            srv.submit(robots[0], worlds[0].x_start)    # second while the first is queued
        wait_all(srv, 1)


@pytest.mark.parametrize("mode", ["lanes", "device_queue"])
def test_size_classes_small_request_passes_large(gpu, mode):
    """Under a size-class policy a small request submitted just after a large
    one completes first: the large class's kernel leaves part of the GPU to
    the small class's lane, so the small request does not wait for it.  The
    timed poll splits each latency into time queued and the batch's device
    time, and reports the class; results stay equal, bit for bit, to the
    same robots alone."""
    big = W.quad2d(4, K=32768, T=100)
    big.obstacles = np.concatenate([big.obstacles] * 12)[:480]
    small = W.unicycle_small(4)
    with gpu.Server(4, 1 << 30, lanes=2) as srv:
        srv.set_policy(small_ops_max=1e9, small_lanes=1, large_share=0.75, shortest_first=True,
                       max_wait_s=0.05, device_queue=mode == "device_queue")
        pol = srv.get_policy()
        assert pol["shortest_first"] and pol["max_wait_s"] == 0.05
        assert pol["lane_classes"] == [0, 1]
        assert pol["device_queue"] == (mode == "device_queue")
        rb = srv.join(big.params, big.obstacles)
        rs = srv.join(small.params, small.obstacles)
        srv.submit(rb, big.x_start)
        time.sleep(0.0005)
        srv.submit(rs, small.x_start)
        got = []
        t0 = time.time()
        while len(got) < 2:
            got += srv.poll_timed()
            assert time.time() - t0 < 60
        assert [d["robot"] for d in got] == [rs, rb], "the small request waited for the large one"
        for d in got:
            assert d["status"] == 0
            assert d["size_class"] == (1 if d["robot"] == rb else 0)
            assert 0.0 <= d["queue"] <= d["latency"] and 0.0 < d["device"] <= d["latency"]
        res = {d["robot"]: d["u0"] for d in got}
        with pytest.raises(gpu.MppiError):          # only while idle
            srv.submit(rs, small.x_start)
            srv.set_policy(small_ops_max=0.0)
        got = []
        while len(got) < 1:
            got += srv.poll_timed()
    for r, w in ((rb, big), (rs, small)):
        with gpu.Batch(2, 1 << 30) as b:
            info = b.slot_info(b.add(w.params, w.obstacles))
        with gpu.Controller(w.params, tiling=dict(samples_per_cta=info["samples_per_cta"], threads=256,
                                                  positions_per_thread=info["positions_per_thread"])) as c:
            c.set_obstacles(w.obstacles)
            c.step(w.x_start)
            np.testing.assert_array_equal(c.get_control(), res[r])


@pytest.mark.parametrize("mode", ["lanes", "device_queue"])
def test_leave_refused_in_flight_and_destroy_with_requests_pending(gpu, mode):
    """A robot cannot leave while its request is queued or running (its slot
    holds the state the request updates), nor can the policy change; once
    the request completes the robot can leave, and a robot that left cannot
    submit.  Destroying the server with requests still queued and running
    returns: the scheduler stops, the resident kernel finishes what it
    claimed and the published rest, and the pool is freed."""
    g = W.rng(21)
    # four planar quadrotors of about 2e10 operations each (about 1 ms of
    # the whole GPU): the last one submitted is still pending when its
    # robot tries to leave
    worlds = [W.quad2d(21 + i, K=16384, T=80) for i in range(4)]
    for w in worlds:
        w.obstacles = W.obstacle_field(g, 300, (0, 0), (20, 10), 0.2, 0.6,
                                       keep_clear=(w.x_start, w.goal))
    srv = gpu.Server(8, 1 << 30, lanes=1)
    try:
        if mode == "device_queue":
            srv.set_policy(small_ops_max=0.0, device_queue=True)
        robots = [srv.join(w.params, w.obstacles) for w in worlds]
        assert all(r is not None for r in robots)
        for r, w in zip(robots, worlds):
            srv.submit(r, w.x_start)
        with pytest.raises(gpu.MppiError) as e:
            srv.leave(robots[-1])
        assert e.value.code == gpu.MPPI_ESTATE
        with pytest.raises(gpu.MppiError) as e:  # the policy changes only while idle
            srv.set_policy(small_ops_max=1e9, device_queue=(mode == "device_queue"))
        assert e.value.code == gpu.MPPI_ESTATE
        got = wait_all(srv, len(robots))
        assert sorted(x[0] for x in got) == sorted(robots)
        assert all(x[4] == 0 for x in got)
        srv.leave(robots[-1])
        with pytest.raises(gpu.MppiError) as e:
            srv.submit(robots[-1], worlds[-1].x_start)
        assert e.value.code == gpu.MPPI_EINVAL
        for r, w in zip(robots[:-1], worlds[:-1]):
            srv.submit(r, w.x_start)
    finally:
        t0 = time.time()
        srv.close()            # with up to three requests pending
        assert time.time() - t0 < 30.0


def test_policy_rejects_bad_values(gpu):
    with gpu.Server(4, 64 << 20, lanes=2) as srv:
        for bad in (dict(small_ops_max=-1.0), dict(small_ops_max=1e9, large_share=0.0),
                    dict(small_ops_max=1e9, large_share=1.5), dict(small_ops_max=1e9, small_lanes=0),
                    dict(small_ops_max=float("nan")), dict(small_ops_max=1e9, max_wait_s=-1.0)):
            with pytest.raises(gpu.MppiError) as e:
                srv.set_policy(**bad)
            assert e.value.code == gpu.MPPI_EINVAL


def test_device_queue_relaunches_for_larger_tiles(gpu):
    """A robot whose tiles need more shared memory than the running resident
    kernel was launched with joins while that kernel works (six long
    requests, about 10 ms of device time, with smaller tiles): the scheduler
    closes the kernel, launches one that fits, and every request completes
    with the same controls as the robot alone."""
    g = W.rng(8)
    longs = []
    for i in range(6):
        w = W.unicycle_stress(20 + i, K=65536, T=60)
        w.obstacles = W.obstacle_field(g, 1000, (0, 0), (50, 50), 0.1, 1.0, keep_clear=(w.x_start, w.goal))
        longs.append(w)
    big = W.quad2d(6, K=8192, T=100)
    with gpu.Server(8, 1 << 30, lanes=2) as srv:
        srv.set_policy(small_ops_max=0.0, device_queue=True)
        robots = [srv.join(w.params, w.obstacles) for w in longs]
        for r, w in zip(robots, longs):
            srv.submit(r, w.x_start)
        time.sleep(0.001)
        rb = srv.join(big.params, big.obstacles)
        srv.submit(rb, big.x_start)
        got = wait_all(srv, len(robots) + 1)
        assert all(d[4] == 0 for d in got)
        res = {d[0]: d[1] for d in got}
        assert srv.stats()["batches"] >= 2   # the kernel was closed and launched again
    for r, w in list(zip(robots, longs)) + [(rb, big)]:
        with gpu.Batch(2, 1 << 30) as b:
            info = b.slot_info(b.add(w.params, w.obstacles))
        with gpu.Controller(w.params, tiling=dict(samples_per_cta=info["samples_per_cta"], threads=256,
                                                  positions_per_thread=info["positions_per_thread"])) as c:
            c.set_obstacles(w.obstacles)
            c.step(w.x_start)
            np.testing.assert_array_equal(c.get_control(), res[r])


def test_server_on_second_device(gpu):
    """A server created while device 1 is current keeps its pool, streams and
    scheduler thread on device 1 (the scheduler thread starts on device 0
    unless it takes the server's device).  Needs two visible GPUs."""
    torch = pytest.importorskip("torch")
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    w = W.unicycle_small(12)
    prev = torch.cuda.current_device()
    try:
        torch.cuda.set_device(1)
        with gpu.Server(4, 64 << 20, lanes=2) as srv:
            r = srv.join(w.params, w.obstacles)
            srv.submit(r, w.x_start)
            (rid, u0, x1, lat, st), = wait_all(srv, 1)
            assert rid == r and st == 0
        with gpu.Batch(2, 64 << 20) as b:
            info = b.slot_info(b.add(w.params, w.obstacles))
        with gpu.Controller(w.params, tiling=dict(samples_per_cta=info["samples_per_cta"], threads=256,
                                                  positions_per_thread=info["positions_per_thread"])) as c:
            c.set_obstacles(w.obstacles)
            c.step(w.x_start)
            np.testing.assert_array_equal(c.get_control(), u0)
    finally:
        torch.cuda.set_device(prev)
