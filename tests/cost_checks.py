"""Per-sample cost tolerance shared by the GPU parity and precision tests.

Costs-to-go are compared at COST_RTOL = 1e-4 relative to max(|S_k|, 1).  A
sample whose rollout passes close to an obstacle has a cost that is
ill-conditioned in its positions: each barrier term 1/h (Eq. 13/15) moves by
2 |p - c| / h^2 per unit of position, and near the boundary that is large.
The step rolls the dynamics out in FP32, in a frame whose origin is the
measured position x0; its positions at distance r from that origin carry an
error of order u r (u = 2^-24: the prefix sums of the increments and the
FP32 representation itself), which no ordering of the arithmetic removes.
So each sample's tolerance is

    COST_RTOL max(|S_k|, 1) + POS_ETA (reach_k + 1 m) sens_k,

where sens_k is the oracle's first-order change of the sample's barrier cost
per unit of position error at every shape point (pinned against finite
differences of the oracle's own cost in test_oracle_pins.py), reach_k is the
rollout's largest distance from x0, and POS_ETA = 8 u.  The test
test_fp32_rollout_error measures the error of an FP32 model of the rollout's
scans at up to about 3.2 u per metre of (reach + 1 m) and checks that POS_ETA
keeps a factor of two over it.  For samples away from the obstacles the
second term is a small fraction of the first, and the bound is the stated
1e-4.
"""
import numpy as np

COST_RTOL = 1e-4
POS_ETA = 8.0 * 2.0 ** -24


def cost_tolerance(ro):
    """Per-sample tolerance on |S_gpu - S_oracle| for the oracle's outputs
    ``ro`` (costs, sens, reach)."""
    S = np.asarray(ro["costs"])
    return COST_RTOL * np.maximum(np.abs(S), 1.0) + POS_ETA * (np.asarray(ro["reach"]) + 1.0) * np.asarray(ro["sens"])


def cost_errors(ro, S_gpu):
    """(largest relative error, number of samples beyond COST_RTOL relative,
    largest ratio of the error to its tolerance, the sample of that ratio)."""
    S = np.asarray(ro["costs"])
    err = np.abs(np.asarray(S_gpu) - S)
    rel = err / np.maximum(np.abs(S), 1.0)
    ratio = err / cost_tolerance(ro)
    k = int(np.argmax(ratio))
    return float(rel.max()), int((rel > COST_RTOL).sum()), float(ratio[k]), k
