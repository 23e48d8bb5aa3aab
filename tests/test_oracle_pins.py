"""Pins for the CPU FP64 oracle: each check compares the oracle with something
other than itself -- an independent library implementation, a closed form,
an invariant, a hand-derived value, or brute force on a tiny input -- so that
a dropped term, a sign or index slip or a transposed operand fails one of
them.  No GPU is needed."""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2504_06437_gb300 import workloads as W


def _cfg(**over):
    """A small unicycle parameter set; tests override what they pin."""
    p = W.base_params(W.UNICYCLE, K=4, T=5, dt=0.1, seed=7)
    p.update(x_goal=np.zeros(3))
    p.update(over)
    return p


# ---------------------------------------------------------------- Philox

_ATEN_PROG = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::philox_engine e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def aten_philox():
    """ATen's header-only Philox4x32-10 engine, compiled and called as an
    independent implementation (key = seed, counter = (offset, subsequence))."""
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    if not os.path.exists(hdr) or shutil.which("g++") is None:
        pytest.skip("ATen Philox header or g++ unavailable")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "p.cpp")
    exe = os.path.join(d, "p")
    with open(src, "w") as f:
        f.write(_ATEN_PROG)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe], check=True)

    def run(triples):
        inp = "\n".join(f"{a} {b} {c}" for a, b, c in triples) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return np.array([[int(v) for v in line.split()] for line in out.strip().splitlines()],
                        dtype=np.uint64)
    yield run
    shutil.rmtree(d, ignore_errors=True)


def test_philox_matches_aten(orc, aten_philox):
    g = np.random.default_rng(1)
    ctrs = g.integers(0, 2**32, size=(300, 4), dtype=np.uint64)
    keys = g.integers(0, 2**32, size=(300, 2), dtype=np.uint64)
    ctrs[:3] = [[0, 0, 0, 0], [2**32 - 1] * 4, [5, 17, 3, 0]]
    keys[:3] = [[0, 0], [2**32 - 1] * 2, [123, 0]]
    triples = [(int(k[0] | (k[1] << 32)), int(c[2] | (c[3] << 32)), int(c[0] | (c[1] << 32)))
               for c, k in zip(ctrs, keys)]
    ref = aten_philox(triples)
    mine = np.array([orc.philox4x32_10(c, k) for c, k in zip(ctrs, keys)], dtype=np.uint64)
    np.testing.assert_array_equal(mine, ref)


def test_philox_counter_sensitivity(orc):
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(orc.philox4x32_10(c, [5, 6]), base)
    assert not np.array_equal(orc.philox4x32_10([1, 2, 3, 4], [5, 7]), base)


# ---------------------------------------------------------------- uniforms

def test_uniform_exact_and_open_interval(orc):
    assert orc.uniform(0) == 2.0**-24
    assert orc.uniform(0xFFFFFFFF) == 1.0 - 2.0**-24
    g = np.random.default_rng(2)
    for r in g.integers(0, 2**32, size=2000):
        u = orc.uniform(int(r))
        m = u * 2**24
        assert m == int(m) and int(m) % 2 == 1        # odd multiple of 2^-24
        assert np.float32(u) == u                     # exact in float32
        assert int(m) >> 1 == int(r) >> 9             # carries the top 23 bits


# ---------------------------------------------------------------- NLN noise (Eq. 11)

def test_box_muller_normals(orc):
    scipy_stats = pytest.importorskip("scipy.stats")
    p = _cfg(ln_sigma=0.0, ln_mu=0.0, sigma=[1.0, 0.0, 0.0, 1.0])
    _, z = orc.noise_batch(p, 1.0, 2000, 50, 3)
    zz = z.reshape(-1, 4)
    N = zz.shape[0]
    for c in range(4):
        col = zz[:, c]
        assert abs(col.mean()) < 5 / math.sqrt(N)
        assert abs(col.var() - 1.0) < 5 * math.sqrt(2.0 / N)
        assert scipy_stats.kstest(col[:20000], "norm").pvalue > 1e-3
    # the two halves of each Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 5 / math.sqrt(N)


def test_nln_reduces_to_gaussian_when_sigma_ln_zero(orc):
    p = _cfg(ln_sigma=0.0, ln_mu=0.0, sigma=[0.3, 0.0, 0.0, 0.7])
    S_e = 0.4
    du, z = orc.noise_batch(p, S_e, 16, 8, 11)
    np.testing.assert_allclose(du[..., 0], math.sqrt(S_e * 0.3) * z[..., 0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(du[..., 1], math.sqrt(S_e * 0.7) * z[..., 1], rtol=1e-15, atol=0)


@pytest.mark.parametrize("ln_mu,ln_sigma", [(0.0, 0.3), (0.2, 0.5)])
def test_nln_moments_eq11(orc, ln_mu, ln_sigma):
    """Eq. 11 with mu_n = 0: mean 0, variance sigma_n^2 exp(2 mu_ln + 2 sigma_ln^2);
    S_e scales the covariance of the normal factor (NLN(0, S_e Sigma))."""
    s00, s11 = 0.5, 0.2
    S_e = 1.7
    p = _cfg(ln_mu=ln_mu, ln_sigma=ln_sigma, sigma=[s00, 0.0, 0.0, s11])
    du, _ = orc.noise_batch(p, S_e, 4000, 100, 0)
    d = du.reshape(-1, 2)
    N = d.shape[0]
    for col, s in ((0, s00), (1, s11)):
        var = S_e * s * math.exp(2 * ln_mu + 2 * ln_sigma**2)
        fourth = 3 * (S_e * s) ** 2 * math.exp(4 * ln_mu + 8 * ln_sigma**2)
        se_var = math.sqrt((fourth - var**2) / N)
        assert abs(d[:, col].mean()) < 5 * math.sqrt(var / N)
        assert abs(d[:, col].var() - var) < 5 * se_var


def test_nln_correlated_sigma(orc):
    """Non-diagonal Sigma: the normal factor is chol(S_e Sigma) z, the
    log-normal factors are independent per element, so
    Cov(du0, du1) = S_e Sigma01 E[g]^2 with E[g] = exp(mu + sigma^2 / 2)."""
    Sig = np.array([[0.5, 0.3], [0.3, 0.4]])
    ln_mu, ln_sigma, S_e = 0.0, 0.3, 1.0
    p = _cfg(ln_mu=ln_mu, ln_sigma=ln_sigma, sigma=Sig.ravel())
    du, _ = orc.noise_batch(p, S_e, 4000, 100, 5)
    d = du.reshape(-1, 2)
    Eg = math.exp(ln_mu + ln_sigma**2 / 2)
    cov = np.mean(d[:, 0] * d[:, 1])
    assert abs(cov - S_e * Sig[0, 1] * Eg**2) < 0.01
    # and the pure-normal case reproduces Sigma exactly in expectation
    p0 = _cfg(ln_mu=0.0, ln_sigma=0.0, sigma=Sig.ravel())
    d0 = orc.noise_batch(p0, S_e, 4000, 100, 5)[0].reshape(-1, 2)
    np.testing.assert_allclose(np.cov(d0.T, bias=True), S_e * Sig, atol=0.01)


# ---------------------------------------------------------------- dynamics (Eq. 1, Eq. 12)

def test_unicycle_constant_control_closed_form(orc):
    """Euler with constant (v, w): x_k = x0 + v dt sum_{j<k} cos(th0 + j a),
    a = w dt, summed in closed form (Dirichlet kernel)."""
    dt, v, w = 0.05, 1.3, 0.7
    p = _cfg(dt=dt, T=40)
    x0 = np.array([0.4, -1.2, 0.3])
    X = orc.simulate(p, x0, np.tile([v, w], (40, 1)))
    a = w * dt
    for k in range(41):
        if k == 0:
            sx = sy = 0.0
        else:
            D = math.sin(k * a / 2) / math.sin(a / 2)
            sx = D * math.cos(x0[2] + (k - 1) * a / 2)
            sy = D * math.sin(x0[2] + (k - 1) * a / 2)
        np.testing.assert_allclose(X[k], [x0[0] + v * dt * sx, x0[1] + v * dt * sy, x0[2] + k * a],
                                   rtol=0, atol=1e-12)


def _quad_cfg(**over):
    p = W.base_params(W.QUAD2D, K=4, T=5, dt=0.02, seed=3)
    p.update(x_goal=np.zeros(6))
    p.update(over)
    return p


def test_quad_hover_is_fixed_point(orc):
    p = _quad_cfg()
    x0 = np.array([1.0, 5.0, 0.0, 0.0, 0.0, 0.0])
    X = orc.simulate(p, x0, np.zeros((30, 2)))
    np.testing.assert_allclose(X, np.tile(x0, (31, 1)), atol=1e-15)


def test_quad_closed_forms(orc):
    m, I, arm, g, dt = W.QUAD_MASS, W.QUAD_INERTIA, W.QUAD_FRAME / 2, W.GRAVITY, 0.02
    p = _quad_cfg()
    # equal extra thrust, level attitude: vertical uniform acceleration
    u = 0.3
    x0 = np.array([0.5, 2.0, 0.0, 0.4, -0.1, 0.0])
    X = orc.simulate(p, x0, np.tile([u, u], (25, 1)))
    acc = 2 * u / m
    for k in range(26):
        assert X[k, 0] == pytest.approx(x0[0] + k * x0[3] * dt, abs=1e-12)
        assert X[k, 1] == pytest.approx(x0[1] + k * x0[4] * dt + acc * dt**2 * k * (k - 1) / 2, abs=1e-12)
        assert X[k, 4] == pytest.approx(x0[4] + k * acc * dt, abs=1e-12)
    # differential thrust: constant angular acceleration (u2 - u1) arm / I
    u1, u2 = -0.1, 0.2
    X = orc.simulate(p, np.zeros(6), np.tile([u1, u2], (10, 1)))
    alpha = (u2 - u1) * arm / I
    for k in range(11):
        assert X[k, 5] == pytest.approx(k * alpha * dt, abs=1e-12)
        assert X[k, 2] == pytest.approx(alpha * dt**2 * k * (k - 1) / 2, abs=1e-12)
    # fixed tilt, hover thrust: lateral acceleration -g sin(phi), vertical g (cos(phi) - 1)
    phi = 0.2
    X = orc.simulate(p, np.array([0, 0, phi, 0, 0, 0.0]), np.zeros((12, 2)))
    for k in range(13):
        assert X[k, 3] == pytest.approx(-k * g * math.sin(phi) * dt, abs=1e-12)
        assert X[k, 4] == pytest.approx(k * g * (math.cos(phi) - 1) * dt, abs=1e-12)
        assert X[k, 0] == pytest.approx(-g * math.sin(phi) * dt**2 * k * (k - 1) / 2, abs=1e-12)


def _car_cfg(**over):
    p = W.base_params(W.ACKERMANN, K=4, T=5, dt=0.02, seed=3)
    p.update(x_goal=np.zeros(4))
    p.update(over)
    return p


def test_ackermann_straight_constant_acceleration(orc):
    """Eq. 14 with zero steering: the heading stays, v_k = v0 + k a dt and
    x_k = x0 + cos(th0) dt sum_{j<k} v_j = x0 + cos(th0) dt (k v0 + a dt k(k-1)/2)."""
    dt, a = 0.02, 1.5
    p = _car_cfg(dt=dt)
    x0 = np.array([3.0, -2.0, 0.6, 2.0])
    X = orc.simulate(p, x0, np.tile([0.0, a], (30, 1)))
    for k in range(31):
        s = k * x0[3] + a * dt * k * (k - 1) / 2
        np.testing.assert_allclose(X[k], [x0[0] + math.cos(x0[2]) * dt * s,
                                          x0[1] + math.sin(x0[2]) * dt * s,
                                          x0[2], x0[3] + k * a * dt], rtol=0, atol=1e-12)


def test_ackermann_constant_steering_closed_form(orc):
    """Eq. 14 at constant speed and steering: heading rate w = v tan(phi) / L,
    so the position is the unicycle's Dirichlet sum with (v, w)."""
    dt, v, phi, L = 0.02, 4.0, 0.3, W.CAR_WHEELBASE
    p = _car_cfg(dt=dt)
    x0 = np.array([1.0, 2.0, -0.4, v])
    X = orc.simulate(p, x0, np.tile([phi, 0.0], (40, 1)))
    a = v * math.tan(phi) / L * dt
    for k in range(41):
        if k == 0:
            sx = sy = 0.0
        else:
            D = math.sin(k * a / 2) / math.sin(a / 2)
            sx = D * math.cos(x0[2] + (k - 1) * a / 2)
            sy = D * math.sin(x0[2] + (k - 1) * a / 2)
        np.testing.assert_allclose(X[k], [x0[0] + v * dt * sx, x0[1] + v * dt * sy,
                                          x0[2] + k * a, v], rtol=0, atol=1e-11)


def _quad5_cfg(**over):
    p = W.base_params(W.QUAD5, K=4, T=5, dt=0.02, seed=3)
    p.update(x_goal=np.zeros(5))
    p.update(over)
    return p


def test_quad5_hover_is_fixed_point(orc):
    """Eq. 12: level attitude, zero pitch rate and zero thrust deviation
    (thrust m g) leave the state unchanged."""
    p = _quad5_cfg()
    x0 = np.array([1.0, 5.0, 0.0, 0.0, 0.0])
    X = orc.simulate(p, x0, np.zeros((30, 2)))
    np.testing.assert_allclose(X, np.tile(x0, (31, 1)), atol=1e-15)


def test_quad5_closed_forms(orc):
    m, g, dt = W.QUAD_MASS, W.GRAVITY, 0.02
    p = _quad5_cfg()
    # level, extra thrust u: vertical acceleration u / m, horizontal drift
    u = 0.4
    x0 = np.array([0.5, 2.0, 0.0, 0.3, -0.2])
    X = orc.simulate(p, x0, np.tile([0.0, u], (25, 1)))
    for k in range(26):
        assert X[k, 0] == pytest.approx(x0[0] + k * x0[3] * dt, abs=1e-12)
        assert X[k, 1] == pytest.approx(x0[1] + k * x0[4] * dt + (u / m) * dt**2 * k * (k - 1) / 2,
                                        abs=1e-12)
        assert X[k, 4] == pytest.approx(x0[4] + k * (u / m) * dt, abs=1e-12)
    # constant pitch rate, hover thrust: theta_k = k w dt, and the
    # horizontal velocity sums -g sin(theta_j) dt over j < k (Dirichlet form)
    w = 1.5
    X = orc.simulate(p, np.zeros(5), np.tile([w, 0.0], (20, 1)))
    a = w * dt
    for k in range(21):
        assert X[k, 2] == pytest.approx(k * a, abs=1e-12)
        sv = 0.0 if k == 0 else math.sin(k * a / 2) / math.sin(a / 2) * math.sin((k - 1) * a / 2)
        assert X[k, 3] == pytest.approx(-g * dt * sv, abs=1e-11)


# ---------------------------------------------------------------- barrier (Eq. 5, Eq. 13/15)

def test_bsum_single_pair_and_floor(orc):
    p = _cfg(shape=np.zeros((1, 2)), h_eps=1e-3)
    ob = [[0.0, 0.0, 1.0]]
    B, coll, mh = orc.bsum(p, ob, [2.0, 0.0, 0.0])
    assert (B, coll, mh) == (pytest.approx(1 / 3), False, pytest.approx(3.0))
    B, coll, mh = orc.bsum(p, ob, [0.5, 0.0, 0.0])          # inside: h < 0
    assert coll and mh == pytest.approx(-0.75) and B == pytest.approx(1e3)
    B, coll, _ = orc.bsum(p, ob, [1.0, 0.0, 0.0])           # on the boundary
    assert coll and B == pytest.approx(1e3)
    B, coll, _ = orc.bsum(p, [[0, 0, 1], [5, 5, 2]], [3.0, 0.0, 0.0])
    assert not coll and B == pytest.approx(1 / 8 + 1 / (4 + 25 - 4))


def test_bsum_shape_point_rotation(orc):
    """A shape point at body (1, 0) sits at position + (cos th, sin th); a
    point at body (0, 1) at position + (-sin th, cos th)."""
    for body, th, world in (((1.0, 0.0), math.pi / 2, (0.0, 1.0)),
                            ((0.0, 1.0), math.pi / 2, (-1.0, 0.0)),
                            ((1.0, 0.0), math.pi, (-1.0, 0.0))):
        p = _cfg(shape=np.array([body]))
        # obstacle centred on the expected world spot: distance 0, h = -r^2
        ob = [[world[0] + 10.0, world[1], 3.0]]
        _, _, mh = orc.bsum(p, ob, [10.0, 0.0, th])
        assert mh == pytest.approx(-9.0, abs=1e-9)
    p = _cfg(shape=np.array([[0.0, 0.0], [0.2, 0.0]]))
    B, _, _ = orc.bsum(p, [[0.0, 3.0, 1.0]], [0.0, 0.0, math.pi / 2])
    assert B == pytest.approx(1 / 8 + 1 / (2.8**2 - 1))


# ---------------------------------------------------------------- DBaS recursion (Eq. 7) and costs (Eq. 9)

def _frozen(p, v=(0.0, 0.0)):
    """Clamp limits that pin every applied control to v (noise has no effect)."""
    p.update(u_min=list(v), u_max=list(v))
    return p


def test_dbas_hand_derived_two_steps(orc):
    """One obstacle c=(0,0), r=1; robot held at (2,0): h = 3, B = 1/3.  Goal
    (3,0): beta_d = 1/8.  gamma = 1/2.  beta_0 = 1/3 (first call),
    w1 = 1/3 + (1/3 - 1/8)/2 = 7/16, w2 = 1/3 + (7/16 - 1/8)/2 = 47/96,
    S = R_B (w1 + w2) = 89/96 with all other costs off."""
    p = _frozen(_cfg(K=3, T=2, Q=[0, 0, 0], Qf=[0, 0, 0], gamma_ctrl=0.0, C_coll=0.0,
                     R_B=1.0, gamma_bas=0.5, x_goal=[3.0, 0.0, 0.0]))
    ctl = orc.new_controller(p)
    x0 = np.array([2.0, 0.0, 0.0])
    r = orc.step(p, [[0.0, 0.0, 1.0]], x0, np.zeros((3, 3)), ctl)
    np.testing.assert_allclose(r["costs"], 89 / 96, rtol=1e-15)
    assert r["beta_used"] == pytest.approx(1 / 3, rel=1e-15)
    assert r["beta_d"] == pytest.approx(1 / 8, rel=1e-15)
    assert r["CB_star"] == pytest.approx(89 / 96, rel=1e-15)
    # second call from the same place: beta = 1/3 + (1/3 - 1/8)/2 = 7/16
    r2 = orc.step(p, [[0.0, 0.0, 1.0]], x0, np.zeros((3, 3)), ctl)
    assert r2["beta_used"] == pytest.approx(7 / 16, rel=1e-15)


@pytest.mark.parametrize("gamma_b", [0.2, 0.5, 0.9])
def test_dbas_geometric_closed_form(orc, gamma_b):
    """Held still at distance d: w_t = b* + g^t (w0 - b*), b* = (B - g beta_d)/(1 - g);
    S = R_B sum_{t=1..T} w_t."""
    T, R_B, d = 17, 2.5, 1.7
    p = _frozen(_cfg(K=2, T=T, Q=[0, 0, 0], Qf=[0, 0, 0], gamma_ctrl=0.0, C_coll=0.0,
                     R_B=R_B, gamma_bas=gamma_b, x_goal=[0.0, 4.0, 0.0]))
    B = 1 / (d * d - 1)
    bd = 1 / 15.0
    bstar = (B - gamma_b * bd) / (1 - gamma_b)
    w = [bstar + gamma_b**t * (B - bstar) for t in range(1, T + 1)]
    ctl = orc.new_controller(p)
    r = orc.step(p, [[0.0, 0.0, 1.0]], [d, 0.0, 0.0], np.zeros((T + 1, 3)), ctl)
    np.testing.assert_allclose(r["costs"], R_B * sum(w), rtol=1e-13)


def test_dbas_equilibrium_at_goal(orc):
    """At x = x_d with beta = beta_d the barrier state stays at beta_d."""
    T = 6
    p = _frozen(_cfg(K=2, T=T, Q=[0, 0, 0], Qf=[0, 0, 0], gamma_ctrl=0.0, C_coll=0.0,
                     R_B=1.0, x_goal=[2.0, 0.0, 0.0]))
    ctl = orc.new_controller(p)
    r = orc.step(p, [[0.0, 0.0, 1.0]], [2.0, 0.0, 0.0], np.zeros((T + 1, 3)), ctl)
    np.testing.assert_allclose(r["costs"], T / 3.0, rtol=1e-14)


def test_costs_hand_derived_K1_T2(orc):
    """Unicycle at the origin, heading 0, controls pinned to (1, 0), dt = 0.1:
    x1 = (0.1,0,0), x2 = (0.2,0,0), reference 0.
    q = 2 x^2 -> 0.02, 0.08; phi = 5 x2^2 = 0.2;
    control cost gamma u^T (S_e Sigma)^-1 v = 2 * 1 * (1 / (0.5 * 0.25)) * 1 = 16 per step.
    S = 0.02 + 0.08 + 0.2 + 32 = 32.3."""
    p = _frozen(_cfg(K=1, T=2, dt=0.1, Q=[2, 3, 0], Qf=[5, 0, 0], gamma_ctrl=2.0,
                     C_coll=0.0, R_B=1.0, mu_coarse=0.5, sigma=[0.25, 0, 0, 1.0]),
                v=(1.0, 0.0))
    ctl = orc.new_controller(p, u_init=np.tile([1.0, 0.0], (2, 1)))
    assert ctl.S_e == 0.5
    r = orc.step(p, np.zeros((0, 3)), np.zeros(3), np.zeros((3, 3)), ctl)
    assert r["costs"][0] == pytest.approx(32.3, rel=1e-14)
    # second component of Q and the cross terms of Sigma^-1 seen separately
    p2 = _frozen(_cfg(K=1, T=1, dt=0.1, Q=[0, 3, 0], Qf=[0, 0, 0], gamma_ctrl=1.0,
                      C_coll=0.0, mu_coarse=0.0, sigma=[2.0, 1.0, 1.0, 1.0]),
                 v=(1.0, 2.0))
    # nominal u = (0.5, -1) differs from the applied v = (1, 2): the control
    # cost is u^T Sigma^-1 v, not v^T Sigma^-1 v
    ctl = orc.new_controller(p2, u_init=[[0.5, -1.0]])
    assert ctl.S_e == 1.0
    x0 = np.array([0.0, 0.0, math.pi / 2])
    r = orc.step(p2, np.zeros((0, 3)), x0, np.zeros((2, 3)), ctl)
    Minv = np.linalg.inv(np.array([[2.0, 1.0], [1.0, 1.0]]))
    y1 = 0.1 * 1.0
    expect = 3 * y1**2 + np.array([0.5, -1.0]) @ Minv @ np.array([1.0, 2.0])
    assert r["costs"][0] == pytest.approx(expect, rel=1e-13)


def test_rollout_cost_matches_closed_form_trajectory(orc):
    """Controls pinned to a constant (v, w); the trajectory has the Dirichlet
    closed form, so S = sum_t q(x_t) + phi(x_T) + control cost can be written
    without the oracle's Euler loop."""
    T, dt, v, w = 20, 0.05, 1.1, -0.6
    g = np.random.default_rng(4)
    xref = g.normal(size=(T + 1, 3))
    Q, Qf = np.array([1.5, 0.7, 0.2]), np.array([4.0, 3.0, 0.5])
    p = _frozen(_cfg(K=2, T=T, dt=dt, Q=Q, Qf=Qf, gamma_ctrl=0.5, C_coll=0.0, R_B=0.0,
                     mu_coarse=0.4, sigma=[0.5, 0, 0, 0.5]), v=(v, w))
    U = np.tile([v, w], (T, 1))
    ctl = orc.new_controller(p, u_init=U)
    x0 = np.array([0.3, 0.1, 0.25])
    r = orc.step(p, np.zeros((0, 3)), x0, xref, ctl)
    a = w * dt
    X = np.zeros((T + 1, 3))
    for k in range(T + 1):
        D = math.sin(k * a / 2) / math.sin(a / 2) if k else 0.0
        X[k] = [x0[0] + v * dt * D * math.cos(x0[2] + (k - 1) * a / 2),
                x0[1] + v * dt * D * math.sin(x0[2] + (k - 1) * a / 2), x0[2] + k * a]
    E = X - xref
    S = np.sum((E[1:] ** 2) @ Q) + (E[T] ** 2) @ Qf
    S += T * 0.5 * (v * v + w * w) / (0.4 * 0.5)
    np.testing.assert_allclose(r["costs"], S, rtol=1e-12)


def test_collision_indicator(orc):
    """Pinned path x_t = (t dt v, 0): an obstacle astride the path collides
    exactly at the steps inside it and adds C_coll for each."""
    T, dt, v = 10, 0.1, 1.0
    p = _frozen(_cfg(K=1, T=T, dt=dt, Q=[0, 0, 0], Qf=[0, 0, 0], gamma_ctrl=0.0,
                     C_coll=100.0, R_B=0.0), v=(v, 0.0))
    ctl = orc.new_controller(p, u_init=np.tile([v, 0.0], (T, 1)))
    ob = [[0.55, 0.0, 0.22]]        # covers x in (0.33, 0.77): steps 4..7
    r = orc.step(p, ob, np.zeros(3), np.zeros((T + 1, 3)), ctl)
    assert r["coll"][0] == 1
    assert r["costs"][0] == pytest.approx(4 * 100.0)
    assert r["minh"][0] == pytest.approx(-0.22**2 + 0.05**2, abs=1e-12)
    ctl = orc.new_controller(p, u_init=np.tile([v, 0.0], (T, 1)))
    r = orc.step(p, [[0.55, 1.0, 0.22]], np.zeros(3), np.zeros((T + 1, 3)), ctl)
    assert r["coll"][0] == 0 and r["costs"][0] == 0.0


# ---------------------------------------------------------------- weights and update (Eq. 4)

def test_weights_invariants(orc):
    g = np.random.default_rng(5)
    S = g.normal(50, 10, size=1000)
    w, rho, Z = orc.weights(S, 3.0)
    assert rho == S.min()
    assert abs(w.sum() - 1) < 1e-14
    w2, _, _ = orc.weights(S + 1234.5, 3.0)
    np.testing.assert_allclose(w2, w, rtol=1e-9, atol=1e-300)
    perm = g.permutation(S.size)
    w3, _, _ = orc.weights(S[perm], 3.0)
    np.testing.assert_allclose(w3, w[perm], rtol=1e-13)
    w0, _, _ = orc.weights(S, 1e-8)
    assert w0[np.argmin(S)] == 1.0 and np.count_nonzero(w0) == 1
    winf, _, _ = orc.weights(S, 1e12)
    np.testing.assert_allclose(winf, 1.0 / S.size, rtol=1e-9)
    wt, _, _ = orc.weights(np.array([3.0, 1.0, 1.0, 7.0]), 1e-8)   # tie splits evenly
    np.testing.assert_allclose(wt, [0, 0.5, 0.5, 0])


def test_weights_brute_force_small(orc):
    """w_i = 1 / sum_j exp((S_i - S_j) / lambda): no min shift, another formula."""
    g = np.random.default_rng(6)
    for K in range(1, 9):
        S = g.normal(5, 2, size=K)
        lam = float(g.uniform(0.3, 4))
        w, _, _ = orc.weights(S, lam)
        bf = np.array([1.0 / sum(math.exp((S[i] - S[j]) / lam) for j in range(K)) for i in range(K)])
        np.testing.assert_allclose(w, bf, rtol=1e-13)


@pytest.mark.parametrize("model", [W.UNICYCLE, W.QUAD2D, W.ACKERMANN, W.QUAD5])
def test_step_update_brute_force(orc, model):
    """Full iteration at K <= 8: du_eff must be clamp(U + NLN draw) - U for the
    same counter, and U* = clamp(U + sum_k w_k du_eff_k) recomputed with
    explicit loops and the brute-force weights; then the shift."""
    w = {W.UNICYCLE: W.unicycle_small, W.QUAD2D: W.quad2d, W.ACKERMANN: W.ackermann,
         W.QUAD5: W.quad5}[model](3)
    p = dict(w.params)
    p.update(K=8, T=6)
    g = np.random.default_rng(8)
    U0 = g.uniform(-0.5, 0.5, size=(6, 2))
    ctl = orc.new_controller(p, u_init=U0)
    x0 = w.x_start.copy()
    r = orc.step(p, w.obstacles, x0, w.reference(x0)[:7], ctl, want_du=True)
    lo, hi = np.array(p["u_min"]), np.array(p["u_max"])
    for k in range(8):
        for t in range(6):
            du, _ = orc.noise(p, 0.4, k, t, 0)
            np.testing.assert_allclose(r["du_eff"][k, t], np.clip(U0[t] + du, lo, hi) - U0[t],
                                       rtol=0, atol=1e-15)
    S = r["costs"]
    lam = p["lambda"]
    bf = np.array([1.0 / sum(math.exp((S[i] - S[j]) / lam) for j in range(8)) for i in range(8)])
    Us = np.zeros((6, 2))
    for t in range(6):
        for d in range(2):
            acc = 0.0
            for k in range(8):
                acc += bf[k] * r["du_eff"][k, t, d]
            Us[t, d] = min(max(U0[t, d] + acc, lo[d]), hi[d])
    np.testing.assert_allclose(r["Ustar"], Us, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["u0"], Us[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["U_next"][:-1], r["Ustar"][1:], rtol=0, atol=0)
    np.testing.assert_array_equal(r["U_next"][-1], r["Ustar"][-1])
    assert ctl.iter == 1 and not ctl.first


def test_lambda_limits_on_update(orc):
    """lambda -> 0: U* = clamp(U + du_eff of the argmin sample);
    lambda -> inf: U* = clamp(U + mean du_eff)."""
    w = W.unicycle_small(1)
    base = dict(w.params)
    base.update(K=64, T=8)
    x0 = w.x_start.copy()
    for lam in (1e-9, 1e12):
        p = dict(base)
        p["lambda"] = lam
        ctl = orc.new_controller(p)
        r = orc.step(p, w.obstacles, x0, w.reference(x0)[:9], ctl, want_du=True)
        lo, hi = np.array(p["u_min"]), np.array(p["u_max"])
        if lam < 1:
            expect = np.clip(r["du_eff"][np.argmin(r["costs"])], lo, hi)
        else:
            expect = np.clip(r["du_eff"].mean(axis=0), lo, hi)
        np.testing.assert_allclose(r["Ustar"], expect, rtol=0, atol=1e-9)


# ------------------------------------------- Savitzky-Golay (Algorithm 1)

@pytest.mark.parametrize("window,order", [(3, 0), (3, 1), (5, 2), (5, 3), (7, 2), (7, 4),
                                          (11, 3), (11, 6), (21, 4), (21, 6)])
def test_sgf_matches_scipy_interp(orc, window, order):
    """Against scipy.signal.savgol_filter's 'interp' mode (least-squares fit
    of the first / last window at the ends), an independent implementation,
    at T = window, window + 1 and 40."""
    signal = pytest.importorskip("scipy.signal")
    g = np.random.default_rng(window * 10 + order)
    for T in sorted({window, window + 1, 40}):
        y = g.normal(size=(T, 2))
        np.testing.assert_allclose(orc.sgf(y, window, order),
                                   signal.savgol_filter(y, window, order, axis=0, mode="interp"),
                                   rtol=0, atol=1e-9)


@pytest.mark.parametrize("window,order,num,den", [
    (5, 2, [-3, 12, 17, 12, -3], 35),
    (7, 2, [-2, 3, 6, 7, 6, 3, -2], 21),
    (9, 2, [-21, 14, 39, 54, 59, 54, 39, 14, -21], 231),
    (7, 4, [5, -30, 75, 131, 75, -30, 5], 231),
    (5, 3, [-3, 12, 17, 12, -3], 35),   # odd order adds nothing at the centre
])
def test_sgf_classic_convolution_coefficients(orc, window, order, num, den):
    """Away from the ends the filter is a convolution whose weights are the
    classic Savitzky-Golay smoothing coefficients (Savitzky and Golay,
    Anal. Chem. 36 (1964), smoothing tables): the response to a unit impulse
    at t0 read over the window around it."""
    T, t0, h = 31, 15, window // 2
    y = np.zeros(T)
    y[t0] = 1.0
    out = orc.sgf(y, window, order)
    np.testing.assert_allclose(out[t0 - h:t0 + h + 1], np.array(num) / den, rtol=0, atol=1e-14)
    assert np.all(out[:t0 - h] == 0) and np.all(out[t0 + h + 1:] == 0)


@pytest.mark.parametrize("window,order", [(3, 1), (5, 2), (9, 4), (21, 6), (63, 6), (63, 3)])
def test_sgf_reproduces_polynomials(orc, window, order):
    """A polynomial of degree <= order is its own least-squares fit, so the
    filter returns it unchanged at every t, the ends included."""
    g = np.random.default_rng(order)
    for T in (window, window + 2, 80):
        t = np.arange(T) / T
        y = np.stack([np.polyval(g.normal(size=order + 1), t) for _ in range(2)], axis=1)
        np.testing.assert_allclose(orc.sgf(y, window, order), y, rtol=0, atol=1e-12)


def test_sgf_full_order_is_identity_and_order_zero_is_mean(orc):
    """order = window - 1 interpolates (identity); order 0 is the moving
    average inside and the mean of the first / last window at the ends."""
    g = np.random.default_rng(5)
    y = g.normal(size=(23, 2))
    np.testing.assert_allclose(orc.sgf(y, 7, 6), y, rtol=0, atol=1e-12)
    out = orc.sgf(y, 5, 0)
    for t in range(23):
        s = min(max(t - 2, 0), 23 - 5)
        np.testing.assert_allclose(out[t], y[s:s + 5].mean(axis=0), rtol=0, atol=1e-15)


def test_step_with_sgf_smooths_the_update(orc):
    """One iteration with the filter on: the sampled costs and weights are
    those of the unfiltered step, and U* = clamp(U + SGF(sum_k w_k du_eff_k))
    with the sums written out and scipy's filter."""
    signal = pytest.importorskip("scipy.signal")
    w = W.quad2d(2)
    p = dict(w.params)
    p.update(K=64, T=15)
    g = np.random.default_rng(9)
    U0 = g.uniform(-0.3, 0.3, size=(15, 2))
    x0 = w.x_start.copy()
    xref = w.reference(x0)[:16]
    r0 = orc.step(p, w.obstacles, x0, xref, orc.new_controller(p, u_init=U0))
    p.update(sgf_window=7, sgf_order=2)
    r = orc.step(p, w.obstacles, x0, xref, orc.new_controller(p, u_init=U0), want_du=True)
    np.testing.assert_array_equal(r["costs"], r0["costs"])
    np.testing.assert_array_equal(r["weights"], r0["weights"])
    dU = np.zeros((15, 2))
    for k in range(64):
        dU += r["weights"][k] * r["du_eff"][k]
    lo, hi = np.array(p["u_min"]), np.array(p["u_max"])
    expect = np.clip(U0 + signal.savgol_filter(dU, 7, 2, axis=0, mode="interp"), lo, hi)
    np.testing.assert_allclose(r["Ustar"], expect, rtol=0, atol=1e-12)
    assert np.abs(r["Ustar"] - r0["Ustar"]).max() > 1e-6  # the filter did act


@pytest.mark.parametrize("window,order", [(4, 1), (17, 2), (5, 5), (9, 7), (-1, 0)])
def test_step_rejects_bad_sgf(orc, window, order):
    p = _cfg(K=4, T=15, sgf_window=window, sgf_order=order)
    with pytest.raises(ValueError):
        orc.step(p, np.zeros((0, 3)), np.zeros(3), np.zeros((16, 3)), orc.new_controller(p))


# ------------------------------------------------ grid map (Sec. V-C)

def _grid_cfg(f, ox=-2.0, oy=1.0, res=0.5, nx=9, ny=7, **over):
    X, Y = np.meshgrid(ox + res * np.arange(nx), oy + res * np.arange(ny))
    g = f(X, Y).astype(np.float32)
    assert np.array_equal(g.astype(np.float64), f(X, Y)), "samples must be exact in float32"
    return _cfg(grid=g, grid_ox=ox, grid_oy=oy, grid_res=res, **over)


def test_grid_bilinear_exact_on_affine_fields(orc):
    """Bilinear interpolation reproduces an affine field exactly inside the
    map; beyond it the point's grid coordinates are clamped to the edge."""
    f = lambda x, y: 1.0 + 0.5 * x - 0.25 * y
    cfg = _grid_cfg(f)
    g = np.random.default_rng(3)
    for px, py in g.uniform([-2.0, 1.0], [2.0, 4.0], size=(50, 2)):
        assert orc.grid_h(cfg, px, py) == pytest.approx(f(px, py), abs=1e-13)
    for px, py in [(-7.0, 2.0), (9.0, 3.3), (0.3, -4.0), (1.1, 20.0), (-9.0, -9.0)]:
        cx, cy = min(max(px, -2.0), 2.0), min(max(py, 1.0), 4.0)
        assert orc.grid_h(cfg, px, py) == pytest.approx(f(cx, cy), abs=1e-13)


def test_grid_quadratic_interpolation_error_and_nodes_match_circle(orc):
    """A grid sampled from the circle barrier h = (x-cx)^2 + (y-cy)^2 - r^2
    returns, between nodes, h + res^2 (fx (1 - fx) + fy (1 - fy)) (linear
    interpolation of a square over a cell of width res), and at nodes the
    grid barrier equals the circle obstacle's barrier exactly."""
    cx, cy, r = 0.5, 2.5, 0.75
    f = lambda x, y: (x - cx) ** 2 + (y - cy) ** 2 - r * r
    cfg = _grid_cfg(f)
    g = np.random.default_rng(4)
    for px, py in g.uniform([-2.0, 1.0], [2.0, 4.0], size=(50, 2)):
        fx = ((px + 2.0) / 0.5) % 1.0
        fy = ((py - 1.0) / 0.5) % 1.0
        expect = f(px, py) + 0.25 * (fx * (1 - fx) + fy * (1 - fy))
        assert orc.grid_h(cfg, px, py) == pytest.approx(expect, abs=1e-12)
    shape = np.array([[0.0, 0.0], [1.0, 0.5]])  # both land on nodes at heading 0
    for x in ([-1.5, 1.5, 0.0], [0.0, 2.0, 0.0], [0.5, 3.0, 0.0]):
        c_grid = dict(cfg, shape=shape)
        c_circ = dict(_cfg(shape=shape))
        bg = orc.bsum(c_grid, np.zeros((0, 3)), x)
        bc = orc.bsum(c_circ, np.array([[cx, cy, r]]), x)
        assert bg[0] == pytest.approx(bc[0], rel=1e-14)
        assert bg[1] == bc[1] and bg[2] == pytest.approx(bc[2], abs=1e-14)


def test_grid_and_circles_add(orc):
    """With both a grid map and circles, the barrier is the sum of the two
    barriers, collided if either collides, min h the smaller."""
    cfg = _grid_cfg(lambda x, y: 0.25 + 0.0 * x + 0.5 * (y - 1.0), shape=[[0.0, 0.0], [0.25, 0.5]])
    circles = np.array([[0.0, 2.0, 0.5], [1.0, 3.0, 0.25]])
    for x in ([0.3, 1.2, 0.4], [-0.2, 2.9, -1.0], [0.9, 3.0, 0.0]):
        both = orc.bsum(cfg, circles, x)
        grid = orc.bsum(cfg, np.zeros((0, 3)), x)
        circ = orc.bsum(dict(cfg, grid=None), circles, x)
        assert both[0] == pytest.approx(grid[0] + circ[0], rel=1e-14)
        assert both[1] == (grid[1] or circ[1])
        assert both[2] == min(grid[2], circ[2])


def test_grid_collision_inside(orc):
    """A shape point where the signed distance is negative collides."""
    cfg = _grid_cfg(lambda x, y: x - 0.5 + 0.0 * y, shape=[[0.0, 0.0]])
    assert orc.bsum(cfg, np.zeros((0, 3)), [0.25, 2.0, 0.0])[1]
    assert not orc.bsum(cfg, np.zeros((0, 3)), [0.75, 2.0, 0.0])[1]


def test_constant_grid_shifts_every_cost_alike(orc):
    """A grid of constant distance c adds P / c to the barrier of every
    state, goal and start included; the DBaS recursion (Eq. 7) is linear in
    that barrier, so every sample's cost moves by the same amount and the
    weights and U* do not change."""
    w = W.ackermann(1)
    p = dict(w.params)
    p.update(K=32, T=10)
    x0 = w.x_start.copy()
    xref = w.reference(x0)[:11]
    r0 = orc.step(p, w.obstacles, x0, xref, orc.new_controller(p))
    g = np.full((4, 5), 2.0, dtype=np.float32)
    pg = dict(p, grid=g, grid_ox=0.0, grid_oy=0.0, grid_res=30.0)
    r1 = orc.step(pg, w.obstacles, x0, xref, orc.new_controller(pg))
    d = r1["costs"] - r0["costs"]
    assert np.ptp(d) < 1e-9 * np.abs(r0["costs"]).max() and abs(d[0]) > 1.0
    np.testing.assert_allclose(r1["weights"], r0["weights"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(r1["Ustar"], r0["Ustar"], rtol=0, atol=1e-10)


# ---------------------------------------------------------------- S_e (Eq. 10)

def test_exploration_rate_no_obstacles_equals_mu(orc):
    w = W.unicycle_small(0)
    p = dict(w.params)
    p.update(K=32, mu_coarse=0.37)
    ctl = orc.new_controller(p)
    r = orc.step(p, np.zeros((0, 3)), w.x_start, w.reference(w.x_start), ctl)
    assert r["CB_star"] == 0.0
    assert ctl.S_e == 0.37


def test_exploration_rate_closed_form(orc):
    """Held still near one obstacle: C_B(X*) follows the geometric closed form,
    S_e = mu ln(e + C_B)."""
    T, d, gb, mu = 9, 1.5, 0.5, 0.4
    p = _frozen(_cfg(K=4, T=T, Q=[0, 0, 0], Qf=[0, 0, 0], gamma_ctrl=0.0, C_coll=0.0,
                     R_B=1.0, gamma_bas=gb, mu_coarse=mu, x_goal=[0.0, 9.0, 0.0]))
    B, bd = 1 / (d * d - 1), 1 / 80.0
    bstar = (B - gb * bd) / (1 - gb)
    CB = sum(bstar + gb**t * (B - bstar) for t in range(1, T + 1))
    ctl = orc.new_controller(p)
    r = orc.step(p, [[0.0, 0.0, 1.0]], [d, 0.0, 0.0], np.zeros((T + 1, 3)), ctl)
    assert r["CB_star"] == pytest.approx(CB, rel=1e-13)
    assert ctl.S_e == pytest.approx(mu * math.log(math.e + CB), rel=1e-14)


def test_exploration_rate_floor_when_cb_negative(orc):
    """beta_0 < beta_d makes the DBaS cost negative; S_e is floored at mu."""
    T = 5
    p = _frozen(_cfg(K=2, T=T, Q=[0, 0, 0], Qf=[0, 0, 0], gamma_ctrl=0.0, C_coll=0.0,
                     R_B=1.0, gamma_bas=0.9, mu_coarse=0.4, x_goal=[1.2, 0.0, 0.0]))
    ctl = orc.new_controller(p)
    r = orc.step(p, [[0.0, 0.0, 1.0]], [20.0, 0.0, 0.0], np.zeros((T + 1, 3)), ctl)
    assert r["CB_star"] < 0
    assert ctl.S_e == 0.4


def test_iteration_counter_changes_noise(orc):
    w = W.unicycle_small(0)
    p = dict(w.params)
    p.update(K=16, T=5)
    ctl = orc.new_controller(p)
    x0 = w.x_start
    r1 = orc.step(p, w.obstacles, x0, w.reference(x0)[:6], ctl, want_du=True)
    ctl2 = orc.new_controller(p)
    ctl2.iter = 1
    r2 = orc.step(p, w.obstacles, x0, w.reference(x0)[:6], ctl2, want_du=True)
    assert not np.allclose(r1["du_eff"], r2["du_eff"])


def test_oracle_thread_count_does_not_change_results(orc):
    w = W.quad2d(2, K=96, T=12)
    x0 = w.x_start
    outs = []
    for n in (1, 3):
        orc.set_threads(n)
        ctl = orc.new_controller(w.params)
        outs.append(orc.step(w.params, w.obstacles, x0, w.reference(x0), ctl))
    orc.set_threads(0)
    np.testing.assert_array_equal(outs[0]["costs"], outs[1]["costs"])
    np.testing.assert_array_equal(outs[0]["Ustar"], outs[1]["Ustar"])


# ------------------------- barrier sensitivity behind the per-sample cost tolerance

def _straight_cfg(**over):
    """Every sample drives straight along +x at 1 m/s from the origin (the
    control box is one point, so the draws do not matter), one shape point at
    the body's origin, the goal far away (its barrier does not move)."""
    base = dict(K=3, T=10, dt=0.05, u_min=[1.0, 0.0], u_max=[1.0, 0.0], h_eps=1e-6,
                shape=np.zeros((1, 2)))
    base.update(over)
    p = _cfg(**base)
    p["x_goal"] = np.array([1000.0, 1000.0, 0.0])
    return p


def _sens_by_differences(orc, p, shift_world, obst):
    """-(dS/ds - dS/dbeta0 * dB(x0)/ds) for a translation s of the world along
    x, every term by central differences of the oracle's own outputs; beta0 is
    reached through the carried beta (first = False: beta0 = B(x0) -
    gamma (beta_d - beta), so dS/dbeta0 = (dS/dbeta) / gamma)."""
    x0 = np.zeros(3)
    xref = np.zeros((p["T"] + 1, 3))

    def cost(s=0.0, beta=0.0):
        q, ob = shift_world(p, obst, s)
        ctl = orc.new_controller(q)
        ctl.first = False
        ctl.beta = beta
        return orc.step(q, ob, x0, xref, ctl)

    d = 1e-5
    dS = (cost(d)["costs"] - cost(-d)["costs"]) / (2 * d)
    g = float(p["gamma_bas"])
    if g > 0:
        dS_dbeta0 = (cost(beta=d)["costs"] - cost(beta=-d)["costs"]) / (2 * d) / g
        qa, oa = shift_world(p, obst, d)
        qb, ob_ = shift_world(p, obst, -d)
        dB0 = (orc.bsum(qa, oa, x0)[0] - orc.bsum(qb, ob_, x0)[0]) / (2 * d)
        dS = dS - dS_dbeta0 * dB0
    return -dS, cost()


def _shift_circles(p, obst, s):
    ob = np.array(obst, dtype=np.float64).copy()
    ob[:, 0] += s
    return p, ob


@pytest.mark.parametrize("gamma, R_B", [(0.0, 1.0), (0.5, 2.0), (1.0, 0.3)])
def test_barrier_sensitivity_is_the_cost_derivative_along_the_line(orc, gamma, R_B):
    """Circles ahead on the line of motion: every barrier gradient along the
    rollout points along x, so the sum of their norms (the oracle's sens)
    equals the derivative of the cost-to-go with respect to moving the
    circles along x, less the part that reaches the cost through the
    barrier state at x0.  gamma 0, 0.5 and 1 cover the weights that Eq. 7's
    recursion gives each step's barrier sum (1, a geometric sum, T - t);
    reach is the 10 steps of 0.05 m."""
    p = _straight_cfg(gamma_bas=gamma, R_B=R_B)
    obst = np.array([[2.0, 0.0, 0.5], [3.5, 0.0, 0.3]])
    want, r = _sens_by_differences(orc, p, _shift_circles, obst)
    assert np.all(want > 0)
    np.testing.assert_allclose(r["sens"], want, rtol=1e-6)
    np.testing.assert_allclose(r["reach"], 0.5, rtol=1e-12)


def test_barrier_sensitivity_grid_term_on_a_unit_ramp(orc):
    """A grid map whose field is h = 3 - x (a signed distance with unit
    gradient): moving the map along x moves every h by the same amount, so
    the grid term's sensitivity 1 / h^2 per step is the cost's derivative
    with respect to the map's origin (less the barrier state at x0)."""
    p = _grid_cfg(lambda X, Y: 3.0 - X, K=3, T=10, dt=0.05, u_min=[1.0, 0.0],
                  u_max=[1.0, 0.0], h_eps=1e-6, shape=np.zeros((1, 2)), gamma_bas=0.5)
    p["x_goal"] = np.array([1000.0, 1000.0, 0.0])

    def shift_map(q, obst, s):
        q = dict(q)
        q["grid_ox"] = p["grid_ox"] + s
        return q, obst

    want, r = _sens_by_differences(orc, p, shift_map, np.zeros((0, 3)))
    assert np.all(want > 0)
    np.testing.assert_allclose(r["sens"], want, rtol=1e-6)


def test_barrier_sensitivity_zero_without_obstacles_and_floored_terms(orc):
    """No obstacle, no term; a circle whose h stays below h_eps along the
    whole rollout (the floored B does not move) adds nothing either."""
    p = _straight_cfg(gamma_bas=0.5)
    ctl = orc.new_controller(p)
    r = orc.step(p, np.zeros((0, 3)), np.zeros(3), np.zeros((p["T"] + 1, 3)), ctl)
    np.testing.assert_array_equal(r["sens"], 0.0)
    p = _straight_cfg(gamma_bas=0.5, h_eps=10.0)
    ctl = orc.new_controller(p)
    r = orc.step(p, [[2.0, 0.0, 0.5]], np.zeros(3), np.zeros((p["T"] + 1, 3)), ctl)
    np.testing.assert_array_equal(r["sens"], 0.0)
