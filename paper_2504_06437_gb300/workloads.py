"""Seeded synthetic worlds and parameter presets.

This module only draws inputs: obstacle fields, start and goal poses,
parameter sets and straight-line reference trajectories.  It holds none of
the controller's arithmetic, and both the CUDA path and the CPU oracle are fed
from it.  Every draw uses ``numpy.random.Generator(PCG64(seed))``.

The paper publishes no obstacle layouts (Sec. V gives only counts and radii),
so these fields stand in for its missions:

* ``unicycle_small``: 10 x 10 m field, 10 obstacles, r ~ U(0.3, 0.8) m,
  K=256, T=30, dt=0.05 s (kinematic unicycle, one shape point).
* ``quad2d``: 20 x 10 m corridor, 40 obstacles, r ~ U(0.2, 0.6) m, K=4096,
  T=50, dt=0.02 s, planar quadrotor with seven shape points on its 0.4 m frame
  (Sec. V-A constants: m = 0.5 kg, I = 0.005 kg m^2, g = 9.81, thrust limit
  0.981 N).
* ``unicycle_stress``: 50 x 50 m field, 200 obstacles, r ~ U(0.1, 1.0) m,
  K=65536, T=100.
* ``quad2d_corridor``: ``quad2d`` with six of its circles moved onto the
  flight line just ahead of the start, so that many samples collide.
* ``batch_mix`` / ``serving_mix``: many independent controllers with mixed
  model, K, T and obstacle count.

Obstacles closer than r + 0.5 m to the start or goal are redrawn so both stay
collision-free.  The reference is a point moving from the start towards the
goal at a set speed (``v_ref``, the paper's v_set), clipped at the goal.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

UNICYCLE = 0
QUAD2D = 1
ACKERMANN = 2
QUAD5 = 3

# Planar quadrotor constants printed in Sec. V-A (frame 0.4 m, mass 0.5 kg,
# inertia 0.005 kg m^2, g = 9.81 m/s^2, thrust limit 0.981 N).
QUAD_MASS = 0.5
QUAD_INERTIA = 0.005
QUAD_FRAME = 0.4
GRAVITY = 9.81
QUAD_THRUST_LIMIT = 0.981
QUAD5_PITCH_RATE_LIMIT = 4.0  # rad/s (Sec. V-A)
CAR_LENGTH, CAR_WIDTH = 4.0, 3.0  # footprint rectangle (Sec. V-B)
CAR_WHEELBASE = 2.5  # not printed in the paper: a reading
CAR_STEER_LIMIT, CAR_ACCEL_LIMIT = 1.013, 2.0  # rad, m/s^2 (Sec. V-B)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def state_dim(model: int) -> int:
    return {QUAD2D: 6, ACKERMANN: 4, QUAD5: 5}.get(model, 3)


def quad_shape_points() -> np.ndarray:
    """Seven points spread evenly along the body axis of the 0.4 m frame:
    the two propellers, the centre and the quarter points between them."""
    s = np.arange(-3, 4) * (QUAD_FRAME / 6.0)
    return np.stack([s, np.zeros_like(s)], axis=1)


def car_shape_points() -> np.ndarray:
    """Eight points of the 4 m x 3 m rectangle around the vehicle position:
    its corners and the midpoints of its sides (length along the heading)."""
    a, b = CAR_LENGTH / 2.0, CAR_WIDTH / 2.0
    return np.array([[a, b], [0.0, b], [-a, b], [-a, 0.0],
                     [-a, -b], [0.0, -b], [a, -b], [a, 0.0]])


def obstacle_field(g: np.random.Generator, J: int, lo, hi, r_lo: float,
                   r_hi: float, keep_clear=(), clearance: float = 0.5) -> np.ndarray:
    """J circles (cx, cy, r), centres uniform in the box [lo, hi], radii
    uniform in [r_lo, r_hi]; circles within r + clearance of any point in
    ``keep_clear`` are redrawn."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    out = np.zeros((J, 3))
    for j in range(J):
        for _ in range(10000):
            c = lo + (hi - lo) * g.random(2)
            r = r_lo + (r_hi - r_lo) * g.random()
            if all(np.hypot(*(c - np.asarray(p[:2]))) > r + clearance for p in keep_clear):
                break
        out[j] = (c[0], c[1], r)
    return out


def corridor_obstacles(g: np.random.Generator, J: int, start, goal, shape,
                       along, lateral, r_lo: float, r_hi: float,
                       margin: float = 0.05) -> np.ndarray:
    """J circles (cx, cy, r) placed across the start-goal line: centres at a
    distance uniform in ``along`` from the start along the line and offset
    uniformly within +-``lateral`` across it, radii uniform in [r_lo, r_hi];
    a circle closer than r + margin to a shape point of the body at the
    start pose, or than r + 0.5 to the goal, is redrawn.  These put
    obstacles where the sampled trajectories go, so that many samples
    collide."""
    a = np.asarray(start[:2], dtype=np.float64)
    d = np.asarray(goal[:2], dtype=np.float64) - a
    d /= np.hypot(*d)
    nrm = np.array([-d[1], d[0]])
    th = float(start[2]) if len(start) > 2 else 0.0
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    body = a + np.asarray(shape, dtype=np.float64).reshape(-1, 2) @ R.T
    out = np.zeros((J, 3))
    for j in range(J):
        for _ in range(10000):
            c = a + g.uniform(*along) * d + g.uniform(-lateral, lateral) * nrm
            r = g.uniform(r_lo, r_hi)
            if (np.hypot(*(body - c).T).min() > r + margin
                    and np.hypot(*(c - np.asarray(goal[:2]))) > r + 0.5):
                break
        out[j] = (c[0], c[1], r)
    return out


def base_params(model: int, K: int, T: int, dt: float, seed: int) -> dict:
    """Parameter dict shared by the oracle and the CUDA binding.  Values the
    paper prints are used where it prints them (gamma = 2 for the control
    cost and mu = 0.4, Sec. V-A/B); the rest follow the presets above."""
    p = dict(model=model, K=K, T=T, dt=dt, seed=seed,
             ln_mu=0.0, ln_sigma=0.3, mu_coarse=0.4, gamma_ctrl=2.0,
             gamma_bas=0.5, R_B=1.0, C_coll=1.0e4, h_eps=1.0e-3,
             mass=QUAD_MASS, inertia=QUAD_INERTIA, arm=QUAD_FRAME / 2.0,
             gravity=GRAVITY)
    p["lambda"] = 1.0
    if model == UNICYCLE:
        p.update(sigma=[0.5, 0.0, 0.0, 0.5], Q=[1.0, 1.0, 0.0],
                 Qf=[10.0, 10.0, 0.0], u_min=[-1.0, -2.0], u_max=[2.0, 2.0],
                 shape=np.zeros((1, 2)))
    elif model == ACKERMANN:  # Sec. V-B: Sigma_u, steering and acceleration limits
        p.update(sigma=[0.075, 0.0, 0.0, 2.0], Q=[1.0, 1.0, 0.0, 0.1],
                 Qf=[10.0, 10.0, 0.0, 1.0],
                 u_min=[-CAR_STEER_LIMIT, -CAR_ACCEL_LIMIT],
                 u_max=[CAR_STEER_LIMIT, CAR_ACCEL_LIMIT],
                 shape=car_shape_points(), wheelbase=CAR_WHEELBASE)
    elif model == QUAD5:  # Sec. V-A: Sigma_u, pitch-rate and thrust limits
        p.update(sigma=[0.4, 0.0, 0.0, 0.12], Q=[1.0, 1.0, 0.1, 0.1, 0.1],
                 Qf=[10.0, 10.0, 1.0, 1.0, 1.0],
                 u_min=[-QUAD5_PITCH_RATE_LIMIT, -QUAD_THRUST_LIMIT],
                 u_max=[QUAD5_PITCH_RATE_LIMIT, QUAD_THRUST_LIMIT],
                 shape=quad_shape_points())
    else:
        p.update(sigma=[0.25, 0.0, 0.0, 0.25],
                 Q=[1.0, 1.0, 0.1, 0.1, 0.1, 0.1],
                 Qf=[10.0, 10.0, 1.0, 1.0, 1.0, 1.0],
                 u_min=[-QUAD_THRUST_LIMIT] * 2, u_max=[QUAD_THRUST_LIMIT] * 2,
                 shape=quad_shape_points())
    return p


@dataclass
class World:
    """One controller's synthetic problem: parameters, obstacles, start,
    goal and reference speed."""
    params: dict
    obstacles: np.ndarray
    x_start: np.ndarray
    goal: np.ndarray
    v_ref: float
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return state_dim(self.params["model"])

    def reference(self, x: np.ndarray) -> np.ndarray:
        """(T+1) x n reference: a point leaving the projection of x on the
        start-goal line at speed v_ref, stopping at the goal."""
        return line_reference(self.params, self.x_start, self.goal, x, self.v_ref)


def line_reference(params: dict, start, goal, x, v_ref: float) -> np.ndarray:
    model, T, dt = params["model"], int(params["T"]), float(params["dt"])
    n = state_dim(model)
    a = np.asarray(start[:2], dtype=np.float64)
    b = np.asarray(goal[:2], dtype=np.float64)
    L = float(np.hypot(*(b - a)))
    d = (b - a) / L if L > 0 else np.zeros(2)
    s0 = float(np.clip(np.dot(np.asarray(x[:2]) - a, d), 0.0, L))
    s = np.clip(s0 + v_ref * dt * np.arange(T + 1), 0.0, L)
    ref = np.zeros((T + 1, n))
    ref[:, 0] = a[0] + s * d[0]
    ref[:, 1] = a[1] + s * d[1]
    moving = (s < L).astype(np.float64)
    if model == UNICYCLE:
        ref[:, 2] = math.atan2(d[1], d[0])
    elif model == ACKERMANN:
        ref[:, 2] = math.atan2(d[1], d[0])
        ref[:, 3] = v_ref * moving
    else:  # both quadrotors: velocities in dims 3 and 4
        ref[:, 3] = v_ref * d[0] * moving
        ref[:, 4] = v_ref * d[1] * moving
    return ref


def _goal_state(model: int, xy, heading: float = 0.0) -> np.ndarray:
    g = np.zeros(state_dim(model))
    g[0], g[1] = xy
    if model in (UNICYCLE, ACKERMANN):
        g[2] = heading
    return g


def unicycle_small(seed: int = 0) -> World:
    g = rng(seed)
    p = base_params(UNICYCLE, K=256, T=30, dt=0.05, seed=seed)
    start = np.array([1.0, 1.0, math.pi / 4])
    goal = _goal_state(UNICYCLE, (9.0, 9.0), math.pi / 4)
    obs = obstacle_field(g, 10, (0, 0), (10, 10), 0.3, 0.8, keep_clear=(start, goal))
    p["x_goal"] = goal
    return World(p, obs, start, goal, v_ref=1.0, name="unicycle_small")


def quad2d(seed: int = 0, K: int = 4096, T: int = 50) -> World:
    g = rng(seed)
    p = base_params(QUAD2D, K=K, T=T, dt=0.02, seed=seed)
    start = np.zeros(6)
    start[:2] = (1.0, 5.0)
    goal = _goal_state(QUAD2D, (19.0, 5.0))
    obs = obstacle_field(g, 40, (0, 0), (20, 10), 0.2, 0.6, keep_clear=(start, goal))
    p["x_goal"] = goal
    return World(p, obs, start, goal, v_ref=1.0, name="quad2d")


def unicycle_stress(seed: int = 0, K: int = 65536, T: int = 100) -> World:
    g = rng(seed)
    p = base_params(UNICYCLE, K=K, T=T, dt=0.05, seed=seed)
    p["u_min"], p["u_max"] = [-2.0, -2.0], [4.0, 2.0]
    start = np.array([2.0, 2.0, math.pi / 4])
    goal = _goal_state(UNICYCLE, (48.0, 48.0), math.pi / 4)
    obs = obstacle_field(g, 200, (0, 0), (50, 50), 0.1, 1.0, keep_clear=(start, goal))
    p["x_goal"] = goal
    return World(p, obs, start, goal, v_ref=2.0, name="unicycle_stress")


def quad2d_corridor(seed: int = 0, K: int = 4096, T: int = 50, n_corridor: int = 6) -> World:
    """The ``quad2d`` world with its first ``n_corridor`` circles moved onto
    the flight line 0.7 to 2 m ahead of the hovering start (offsets within
    +-1 m across it, r ~ U(0.2, 0.6) m, clear of the body at the start): the
    sampled trajectories reach them within the horizon, and about 40 % of
    the samples of the first step collide.  Same sizes as ``quad2d``
    (J = 40, P = 7)."""
    w = quad2d(seed, K=K, T=T)
    g = rng(seed + 1001)
    obs = w.obstacles.copy()
    obs[:n_corridor] = corridor_obstacles(g, n_corridor, w.x_start, w.goal, w.params["shape"],
                                          (0.7, 2.0), 1.0, 0.2, 0.6)
    return World(w.params, obs, w.x_start, w.goal, w.v_ref, name="quad2d_corridor")


def _mixed_world(g: np.random.Generator, idx: int, seed: int, K_lo: int,
                 K_hi: int, T_lo: int, T_hi: int, J_lo: int, J_hi: int) -> World:
    model = UNICYCLE if idx % 2 == 0 else QUAD2D
    K = int(math.exp(g.uniform(math.log(K_lo), math.log(K_hi))))
    K = max(32, (K // 32) * 32)
    T = int(g.integers(T_lo, T_hi + 1))
    J = int(g.integers(J_lo, J_hi + 1))
    cseed = seed * 100003 + idx
    if model == UNICYCLE:
        side = 10.0 * math.sqrt(max(J, 10) / 10.0)
        p = base_params(UNICYCLE, K=K, T=T, dt=0.05, seed=cseed)
        start = np.array([1.0, 1.0, math.pi / 4])
        goal = _goal_state(UNICYCLE, (side - 1.0, side - 1.0), math.pi / 4)
        obs = obstacle_field(g, J, (0, 0), (side, side), 0.3, 0.8, keep_clear=(start, goal))
        v_ref = 1.0
    else:
        length = 20.0 * max(1.0, J / 40.0)
        p = base_params(QUAD2D, K=K, T=T, dt=0.02, seed=cseed)
        start = np.zeros(6)
        start[:2] = (1.0, 5.0)
        goal = _goal_state(QUAD2D, (length - 1.0, 5.0))
        obs = obstacle_field(g, J, (0, 0), (length, 10), 0.2, 0.6, keep_clear=(start, goal))
        v_ref = 1.0
    p["x_goal"] = goal
    return World(p, obs, start, goal, v_ref=v_ref, name=f"mix{idx}")


def batch_mix(n: int = 512, seed: int = 0) -> list[World]:
    """Independent controllers, alternating unicycle / quadrotor, with
    K log-uniform in [1024, 16384] (multiple of 32), T uniform in [20, 80]
    and obstacle count uniform in [5, 300]."""
    g = rng(seed)
    return [_mixed_world(g, i, seed, 1024, 16384, 20, 80, 5, 300) for i in range(n)]


def serving_mix(n: int = 1000, seed: int = 0) -> list[World]:
    """Robots for the serving loop: K log-uniform in [512, 32768], T in
    [20, 100], obstacles in [5, 500], alternating models."""
    g = rng(seed)
    return [_mixed_world(g, i, seed, 512, 32768, 20, 100, 5, 500) for i in range(n)]


def ackermann(seed: int = 0, K: int = 1024, T: int = 20, J: int = 5) -> World:
    """The ground-vehicle mission of Sec. V-B in synthetic form: K = M = 1024
    samples, T = N = 20 steps of 0.02 s, J circles of radius 4.3 m along a
    100 m x 30 m corridor, alternately above and below the centre line so
    that the vehicle (4 m x 3 m, 8 shape points) passes narrow gaps, at a
    reference speed of 5 m/s.  The paper publishes no layout."""
    g = rng(seed)
    p = base_params(ACKERMANN, K=K, T=T, dt=0.02, seed=seed)
    start = np.array([5.0, 15.0, 0.0, 0.0])
    goal = _goal_state(ACKERMANN, (95.0, 15.0), 0.0)
    xs = np.sort(g.uniform(20.0, 80.0, J))
    side = np.where(np.arange(J) % 2 == 0, 1.0, -1.0)
    ys = 15.0 + side * g.uniform(5.5, 7.0, J)  # gaps of about 1.2 to 2.7 m each side
    obs = np.stack([xs, ys, np.full(J, 4.3)], axis=1)
    p["x_goal"] = goal
    return World(p, obs, start, goal, v_ref=5.0, name="ackermann")


def quad5(seed: int = 0, K: int = 1024, T: int = 20, J: int = 3) -> World:
    """The quadrotor mission of Sec. V-A with the paper's 5-state model, in
    synthetic form: K = 1024, T = 20 steps of 0.02 s, J circles of radius
    0.8 m along a 20 m x 10 m corridor, alternately above and below the
    flight line, hover start, reference speed 1 m/s."""
    g = rng(seed)
    p = base_params(QUAD5, K=K, T=T, dt=0.02, seed=seed)
    start = np.zeros(5)
    start[:2] = (1.0, 5.0)
    goal = _goal_state(QUAD5, (19.0, 5.0))
    xs = np.sort(g.uniform(5.0, 15.0, J))
    side = np.where(np.arange(J) % 2 == 0, 1.0, -1.0)
    zs = 5.0 + side * g.uniform(1.2, 1.6, J)
    obs = np.stack([xs, zs, np.full(J, 0.8)], axis=1)
    p["x_goal"] = goal
    return World(p, obs, start, goal, v_ref=1.0, name="quad5")


def sdf_grid(discs, boxes, ox: float, oy: float, res: float, nx: int, ny: int) -> np.ndarray:
    """A grid map as a perception stack would hand it over: the exact signed
    distance (m) from each sample (ox + i res, oy + j res) to the union of
    the discs (cx, cy, r) and the axis-aligned boxes (x0, y0, x1, y1),
    negative inside, as an ny x nx float32 array (row j, column i)."""
    X, Y = np.meshgrid(ox + res * np.arange(nx), oy + res * np.arange(ny))
    d = np.full((ny, nx), np.inf)
    for cx, cy, r in np.asarray(discs, dtype=np.float64).reshape(-1, 3):
        d = np.minimum(d, np.hypot(X - cx, Y - cy) - r)
    for x0, y0, x1, y1 in np.asarray(boxes, dtype=np.float64).reshape(-1, 4):
        qx = np.abs(X - 0.5 * (x0 + x1)) - 0.5 * (x1 - x0)
        qy = np.abs(Y - 0.5 * (y0 + y1)) - 0.5 * (y1 - y0)
        outside = np.hypot(np.maximum(qx, 0.0), np.maximum(qy, 0.0))
        d = np.minimum(d, outside + np.minimum(np.maximum(qx, qy), 0.0))
    return d.astype(np.float32)


def ackermann_grid(seed: int = 0, K: int = 1024, T: int = 20, res: float = 0.1) -> World:
    """The vehicle mission with its obstacles given as a grid map instead of
    circles (Sec. V-C: the vehicle plans on a 2D grid map built from its
    LiDAR point cloud).  The circles of the ``ackermann`` preset plus the
    corridor's two walls, rasterised as a signed-distance grid over the
    100 m x 30 m corridor at ``res`` (0.1 m: 1001 x 301 samples); no circle
    obstacles are passed."""
    w = ackermann(seed, K=K, T=T)
    nx, ny = int(round(100.0 / res)) + 1, int(round(30.0 / res)) + 1
    walls = [(-5.0, -5.0, 105.0, 0.5), (-5.0, 29.5, 105.0, 35.0)]
    g = sdf_grid(w.obstacles, walls, 0.0, 0.0, res, nx, ny)
    p = dict(w.params, grid=g, grid_ox=0.0, grid_oy=0.0, grid_res=res)
    return World(p, np.zeros((0, 3)), w.x_start, w.goal, w.v_ref, name="ackermann_grid")


PRESETS = {
    "unicycle_small": unicycle_small,
    "quad2d": quad2d,
    "quad2d_corridor": quad2d_corridor,
    "unicycle_stress": unicycle_stress,
    "ackermann": ackermann,
    "quad5": quad5,
    "ackermann_grid": ackermann_grid,
}
