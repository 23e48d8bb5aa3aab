"""Precision of the GPU step against the FP64 oracle at the three
single-controller workload sizes (unicycle K=256 T=30 J=10, planar quadrotor
K=4096 T=50 J=40 with 7 shape points, unicycle K=65536 T=100 J=200), one step
each from the same inputs, every sample compared, in the launch shape that
bench.py times (the autotuner's pick); and, at the same full sizes, worlds
in which thousands of samples collide, so that the collided-set identity and
the collision cost are checked where the several-wave grids, the
80-register form and the two-level merge run.

The rollout is FP32; the per-sample costs are float pairs relative to a
shared base; the weights, their normaliser and the weighted update are
float-pair sums with log-sum-exp merges.  Each case prints one line
``PRECISION {json}`` (run with -s to see it) with the maximum and 99th
percentile relative cost error, the maximum absolute error of U* and of the
weights, the relative error of the next exploration rate S_e, the number of
collided samples, and the collided-set mismatches away from h = 0 (samples
whose smallest |h| is within H_MARGIN are near-ties, counted separately),
the number of samples beyond 1e-4 relative cost error and the largest ratio
of a cost error to its tolerance; it asserts the tolerances (1e-4 relative
cost, widened for samples that pass close to an obstacle by what the FP32
rollout's positions allow: cost_checks; 1e-5 absolute U*; identical
collided set away from near-ties)."""
import json

import numpy as np
import pytest

from paper_2504_06437_gb300 import workloads as W
from cost_checks import cost_errors
from weight_checks import SELF_RTOL, weight_errors

pytestmark = pytest.mark.gpu

U_ATOL = 1e-5
H_MARGIN = 1e-4


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06437_gb300 import binding
    binding.load()
    return binding


# Worlds in which many samples collide, at the full bench sizes (Algorithm 1's
# collision indicator): the stress world (K 65536, T 100, J 200) from a
# nominal sequence that turns at 0.5 rad/s at 1 m/s, which grazes the circle
# 2.3 m ahead of the start (about 6000 samples collide), and at -0.5 rad/s,
# which runs into it (about 40000); the quadrotor world with six circles on
# its flight line (about 1700 of 4096).  (name, preset, nominal u, least
# number of collided samples the case must reach)
COLLIDING = {
    "unicycle_stress_graze": ("unicycle_stress", (1.0, 0.5), 2000),
    "unicycle_stress_hit": ("unicycle_stress", (1.0, -0.5), 20000),
    "quad2d_corridor": ("quad2d_corridor", None, 1000),
}


def _case(name):
    if name in COLLIDING:
        preset, u, _ = COLLIDING[name]
        w = W.PRESETS[preset](0)
        U = None if u is None else np.tile(np.asarray(u, dtype=np.float64), (int(w.params["T"]), 1))
        return w, U
    return W.PRESETS[name](0), None


@pytest.mark.parametrize("name", ["unicycle_small", "quad2d", "unicycle_stress", "ackermann", "quad5",
                                  *COLLIDING])
def test_precision_against_oracle(gpu, orc, name):
    """In the launch shape bench.py times for the workload (the autotuner's
    pick)."""
    w, u_init = _case(name)
    p = w.params
    ctl = orc.new_controller(p, u_init)
    x = w.x_start
    xref = w.reference(x)
    ro = orc.step(p, w.obstacles, x, xref, ctl)
    tiling, _ = gpu.autotune(p, w.obstacles, iters=10, flush_bytes=256 << 20)
    with gpu.Controller(p, u_init=u_init, tiling=tiling) as g:
        g.set_obstacles(w.obstacles)
        g.step(x, xref)
        u0, _ = g.get_control(want_U=True)
        dbg = g.get_debug()
        regs = g.kernel_regs()
    rec = _compare(name, w, ro, ctl, u0, dbg, tiling, regs)
    if name in COLLIDING:
        assert rec["collided"] >= COLLIDING[name][2], rec["collided"]


def test_precision_largest_K(gpu, orc):
    """K at its limit (2^22 samples; T 8, the stress world's eight first
    circles), in the library's default launch shape: the tiles form 64
    groups of thousands of rows each, more than the merging CTA has
    threads, so each thread of a group merge scales several source rows.
    Every sample compared, as above."""
    w = W.unicycle_stress(0, K=1 << 22, T=8)
    w.obstacles = w.obstacles[:8]
    p = w.params
    ctl = orc.new_controller(p)
    x = w.x_start
    xref = w.reference(x)
    ro = orc.step(p, w.obstacles, x, xref, ctl)
    with gpu.Controller(p) as g:
        g.set_obstacles(w.obstacles)
        g.step(x, xref)
        u0, _ = g.get_control(want_U=True)
        dbg = g.get_debug()
        regs = g.kernel_regs()
        tiling = g.tiling()
    n_tiles = tiling["n_ctas"]
    assert -(-n_tiles // 64) > tiling["threads"], tiling  # group rows > threads
    _compare("unicycle_largest_K", w, ro, ctl, u0, dbg, tiling, regs)


def _compare(name, w, ro, ctl, u0, dbg, tiling, regs):
    """Checks one GPU step against the oracle's and prints its PRECISION line."""
    p = w.params
    rel = np.abs(dbg["costs"] - ro["costs"]) / np.maximum(np.abs(ro["costs"]), 1.0)
    _, beyond, tol_ratio, _ = cost_errors(ro, dbg["costs"])
    u_err = float(np.abs(dbg["Ustar"] - ro["Ustar"]).max())
    w_err, w_self, w_ratio = weight_errors(ro, dbg, float(p["lambda"]))
    sure = np.abs(ro["minh"]) > H_MARGIN
    mismatch = int(np.sum((ro["coll"] != dbg["coll"]) & sure))
    rec = dict(workload=name, K=int(p["K"]), T=int(p["T"]), J=int(w.obstacles.shape[0]),
               tiling=[tiling["samples_per_cta"], tiling["threads"], tiling["positions_per_thread"]],
               kernel_regs=regs,
               cost_rel_max=float(rel.max()), cost_rel_p99=float(np.quantile(rel, 0.99)),
               cost_beyond_rtol=beyond, cost_tolerance_ratio=tol_ratio,
               u_star_abs_max=u_err, u0_abs_max=float(np.abs(u0 - ro["u0"]).max()),
               weight_abs_max=w_err, weight_self_rel_max=w_self, weight_allowance_ratio=w_ratio,
               weight_sum_minus_1=float(dbg["weights"].sum() - 1.0),
               S_e_next_rel=float(abs(dbg["S_e_next"] - ctl.S_e) / ctl.S_e),
               collided=int(ro["coll"].sum()), collided_mismatch=mismatch,
               near_ties=int(np.sum(~sure)))
    print("PRECISION " + json.dumps(rec))
    assert tol_ratio <= 1.0
    assert u_err <= U_ATOL
    assert w_self <= SELF_RTOL
    assert w_ratio <= 1.0
    assert mismatch == 0
    return rec
