"""Precision of the GPU step against the FP64 oracle at the three
single-controller workload sizes (unicycle K=256 T=30 J=10, planar quadrotor
K=4096 T=50 J=40 with 7 shape points, unicycle K=65536 T=100 J=200), one step
each from the same inputs, every sample compared, in the launch shape that
bench.py times (the autotuner's pick).

The rollout is FP32; the per-sample costs are float pairs relative to a
shared base; the weights, their normaliser and the weighted update are
float-pair sums with log-sum-exp merges.  Each case prints one line
``PRECISION {json}`` (run with -s to see it) with the maximum and 99th
percentile relative cost error, the maximum absolute error of U* and of the
weights, the relative error of the next exploration rate S_e, the number of
collided samples, and the collided-set mismatches away from h = 0 (samples
whose smallest |h| is within H_MARGIN are near-ties, counted separately); it
asserts the tolerances (1e-4 relative cost, 1e-5 absolute U*, identical
collided set away from near-ties)."""
import json

import numpy as np
import pytest

from paper_2504_06437_gb300 import workloads as W

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-4
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


@pytest.mark.parametrize("name", ["unicycle_small", "quad2d", "unicycle_stress", "ackermann", "quad5"])
def test_precision_against_oracle(gpu, orc, name):
    """In the launch shape bench.py times for the workload (the autotuner's
    pick)."""
    w = W.PRESETS[name](0)
    p = w.params
    ctl = orc.new_controller(p)
    x = w.x_start
    xref = w.reference(x)
    ro = orc.step(p, w.obstacles, x, xref, ctl)
    tiling, _ = gpu.autotune(p, w.obstacles, iters=10)
    with gpu.Controller(p, tiling=tiling) as g:
        g.set_obstacles(w.obstacles)
        g.step(x, xref)
        u0, _ = g.get_control(want_U=True)
        dbg = g.get_debug()
        regs = g.kernel_regs()
    rel = np.abs(dbg["costs"] - ro["costs"]) / np.maximum(np.abs(ro["costs"]), 1.0)
    u_err = float(np.abs(dbg["Ustar"] - ro["Ustar"]).max())
    w_err = float(np.abs(dbg["weights"] - ro["weights"]).max())
    sure = np.abs(ro["minh"]) > H_MARGIN
    mismatch = int(np.sum((ro["coll"] != dbg["coll"]) & sure))
    rec = dict(workload=name, K=int(p["K"]), T=int(p["T"]), J=int(w.obstacles.shape[0]),
               tiling=[tiling["samples_per_cta"], tiling["threads"], tiling["positions_per_thread"]],
               kernel_regs=regs,
               cost_rel_max=float(rel.max()), cost_rel_p99=float(np.quantile(rel, 0.99)),
               u_star_abs_max=u_err, u0_abs_max=float(np.abs(u0 - ro["u0"]).max()),
               weight_abs_max=w_err, weight_sum_minus_1=float(dbg["weights"].sum() - 1.0),
               S_e_next_rel=float(abs(dbg["S_e_next"] - ctl.S_e) / ctl.S_e),
               collided=int(ro["coll"].sum()), collided_mismatch=mismatch,
               near_ties=int(np.sum(~sure)))
    print("PRECISION " + json.dumps(rec))
    assert rel.max() <= COST_RTOL
    assert u_err <= U_ATOL
    assert mismatch == 0
