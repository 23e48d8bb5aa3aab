"""The position error of an FP32 rollout, against which the per-sample cost
tolerance (cost_checks.POS_ETA) is set.

A model of the step's arithmetic for the kinematic unicycle in numpy: the
heading and the positions are inclusive prefix sums of FP32 increments,
formed 32 steps at a time by a doubling scan (each lane adds the value 1, 2,
4, 8 and 16 lanes back) and carried from one 32-step segment to the next, as
the warp scans do; cosine and sine are taken in FP64 of the FP32 heading and
rounded.  Against the same rollout in FP64 summed in order, over random
100-step rollouts at up to 4 m/s (up to 20 m of reach), the largest position
error per metre of (reach + 1 m) must stay within half of POS_ETA, so that
the tolerance keeps a factor of two over the model."""
import numpy as np

from cost_checks import POS_ETA


def _scan(a):
    """Inclusive FP32 prefix sums in 32-wide doubling scans, carried across
    segments."""
    f = np.float32
    a = a.astype(f)
    out = np.empty_like(a)
    carry = f(0.0)
    for c0 in range(0, len(a), 32):
        n = min(32, len(a) - c0)
        v = np.zeros(32, f)
        v[:n] = a[c0:c0 + n]
        o = 1
        while o < 32:
            v = (v + np.concatenate([np.zeros(o, f), v[:-o]])).astype(f)
            o *= 2
        v = (v + carry).astype(f)
        out[c0:c0 + n] = v[:n]
        carry = v[n - 1]
    return out


def test_fp32_rollout_position_error_within_half_the_tolerance_model():
    rng = np.random.default_rng(0)
    T, dt = 100, 0.05
    f = np.float32
    worst = 0.0
    for _ in range(200):
        v = rng.uniform(0.5, 4.0, T)
        w = rng.uniform(-2.0, 2.0, T)
        th0 = rng.uniform(-np.pi, np.pi)
        th = th0 + np.cumsum(w * dt)
        x = np.cumsum(v * np.cos(th) * dt)
        y = np.cumsum(v * np.sin(th) * dt)
        th32 = (f(th0) + _scan(w.astype(f) * f(dt))).astype(f)
        vdt = (v.astype(f) * f(dt)).astype(f)
        x32 = _scan(vdt * np.cos(th32.astype(np.float64)).astype(f))
        y32 = _scan(vdt * np.sin(th32.astype(np.float64)).astype(f))
        err = np.hypot(x32 - x, y32 - y)
        reach = np.hypot(x, y).max()
        worst = max(worst, err.max() / (reach + 1.0))
    assert 0.0 < worst <= POS_ETA / 2, (worst, POS_ETA)
