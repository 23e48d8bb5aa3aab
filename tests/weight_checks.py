"""Checks of the Eq. 4 weights shared by the GPU parity and precision tests.

w_k = exp(-(S_k - rho) / lambda) / Z.  The GPU path reduces the minimum rho
and the normaliser Z as float pairs; the weights it reports are formed in
FP64 from its own per-sample costs and that rho and Z.  Two checks follow:

* self-consistency: against Eq. 4 written out in FP64 (numpy) from the same
  GPU costs, which isolates the hot path's rho and Z from the rollout's
  rounding: relative error at most SELF_RTOL on every weight above 1e-8;
* against the oracle, within what the measured cost errors explain.  With
  dS_k = S_k(GPU) - S_k(oracle), Eq. 4 moves ln w_k by
  -(dS_k - sum_j w_j dS_j) / lambda to first order (the shift of rho
  cancels, the sum is the change of ln Z), so each weight must satisfy
  |w_gpu - w_oracle| <= W_ATOL + w_oracle (1.5 |dS_k - sum_j w_j dS_j| / lambda
  + W_RTOL): a margin of 1.5 on the propagated error, W_RTOL for the
  float-pair normaliser and the FP32 exponentials of the merges, W_ATOL for
  the weights far below the largest (the mean weight is 1 / K).
"""
import numpy as np

W_ATOL = 1e-6
W_RTOL = 1e-5
SELF_RTOL = 1e-6


def weight_errors(ro, dbg, lam):
    """(max abs error against the oracle, max relative error against Eq. 4
    from the GPU's own costs, worst ratio of the oracle error to its
    allowance) for one step."""
    w_g, w_o, S_g = dbg["weights"], ro["weights"], dbg["costs"]
    e = np.exp(-(S_g - S_g.min()) / lam)
    w_self = e / e.sum()
    big = w_self > 1e-8
    self_rel = float(np.abs(w_g[big] / w_self[big] - 1.0).max())
    dS = S_g - ro["costs"]
    prop = np.abs(dS - np.sum(w_o * dS)) / lam
    err = np.abs(w_g - w_o)
    return float(err.max()), self_rel, float((err / (W_ATOL + w_o * (1.5 * prop + W_RTOL))).max())


def check_weights(ro, dbg, lam, label=""):
    w_abs, self_rel, ratio = weight_errors(ro, dbg, lam)
    assert self_rel <= SELF_RTOL, f"{label} weights off Eq. 4 of the GPU costs by {self_rel:.3e}"
    assert ratio <= 1.0, f"{label} weights off the oracle's by {w_abs:.3e} (allowance ratio {ratio:.2f})"
    return w_abs, self_rel, ratio
