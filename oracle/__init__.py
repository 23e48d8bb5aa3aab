"""CPU FP64 oracle for one DBaS-Log-MPPI iteration (arXiv 2504.06437).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The CUDA product path never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``mppi_oracle.c`` (plain C99, double precision,
compiled with ``-ffp-contract=off`` so x86 and Arm give the same bits).  This
module only compiles it and marshals numpy arrays through ctypes.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, invariants, brute force or an independent library
implementation; the closed-loop mission behaviour of Table I is
"parity unpinned" (the paper gives no obstacle layouts).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mppi_oracle.c")
_LIB = os.path.join(_HERE, "liborc_mppi.so")

UNICYCLE = 0
QUAD2D = 1
ACKERMANN = 2
QUAD5 = 3


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library and return its path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("model", C.c_int32), ("K", C.c_int32), ("T", C.c_int32),
        ("dt", C.c_double), ("lam", C.c_double),
        ("sigma", C.c_double * 4),
        ("ln_mu", C.c_double), ("ln_sigma", C.c_double),
        ("mu_coarse", C.c_double),
        ("gamma_ctrl", C.c_double), ("gamma_bas", C.c_double),
        ("R_B", C.c_double), ("C_coll", C.c_double), ("h_eps", C.c_double),
        ("Q", C.c_double * 6), ("Qf", C.c_double * 6),
        ("u_min", C.c_double * 2), ("u_max", C.c_double * 2),
        ("x_goal", C.c_double * 6),
        ("n_shape", C.c_int32),
        ("shape", C.c_double * 16),
        ("seed", C.c_uint64),
        ("mass", C.c_double), ("inertia", C.c_double),
        ("arm", C.c_double), ("gravity", C.c_double),
        ("wheelbase", C.c_double),
        ("sgf_window", C.c_int32), ("sgf_order", C.c_int32),
        ("grid", C.POINTER(C.c_float)), ("grid_nx", C.c_int32), ("grid_ny", C.c_int32),
        ("grid_ox", C.c_double), ("grid_oy", C.c_double), ("grid_res", C.c_double),
    ]


class _State(C.Structure):
    _fields_ = [("U", C.POINTER(C.c_double)), ("S_e", C.c_double),
                ("beta", C.c_double), ("first", C.c_int32),
                ("iter", C.c_uint64)]


class _Out(C.Structure):
    _fields_ = [
        ("costs", C.POINTER(C.c_double)), ("coll", C.POINTER(C.c_uint8)),
        ("minh", C.POINTER(C.c_double)), ("weights", C.POINTER(C.c_double)),
        ("du_eff", C.POINTER(C.c_double)), ("Ustar", C.POINTER(C.c_double)),
        ("u0", C.POINTER(C.c_double)),
        ("CB_star", C.c_double), ("beta_used", C.c_double),
        ("beta_d", C.c_double), ("rho", C.c_double), ("Z", C.c_double),
        ("sens", C.POINTER(C.c_double)), ("reach", C.POINTER(C.c_double)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        lib.orc_uniform.argtypes = [C.c_uint32]
        lib.orc_uniform.restype = C.c_double
        lib.orc_noise.argtypes = [C.POINTER(_Params), C.c_double, C.c_int32,
                                  C.c_int32, C.c_uint64, dp, dp]
        lib.orc_noise_batch.argtypes = [C.POINTER(_Params), C.c_double,
                                        C.c_int32, C.c_int32, C.c_uint64,
                                        dp, dp]
        lib.orc_dynamics.argtypes = [C.POINTER(_Params), dp, dp, dp]
        lib.orc_bsum.argtypes = [C.POINTER(_Params), dp, C.c_int32, dp, dp,
                                 C.POINTER(C.c_int32), dp]
        lib.orc_simulate.argtypes = [C.POINTER(_Params), dp, dp, dp]
        lib.orc_weights.argtypes = [dp, C.c_int32, C.c_double, dp, dp]
        lib.orc_weights.restype = C.c_double
        lib.orc_step.argtypes = [C.POINTER(_Params), dp, C.c_int32, dp, dp,
                                 C.POINTER(_State), C.POINTER(_Out)]
        lib.orc_step.restype = C.c_int
        lib.orc_sample_costs.argtypes = [C.POINTER(_Params), dp, C.c_int32, dp, dp,
                                         C.POINTER(_State), C.POINTER(C.c_int32), C.c_int32,
                                         dp, C.POINTER(C.c_uint8), dp, dp, dp]
        lib.orc_sample_costs.restype = C.c_int
        lib.orc_grid_h.argtypes = [C.POINTER(_Params), C.c_double, C.c_double]
        lib.orc_grid_h.restype = C.c_double
        lib.orc_sgf.argtypes = [dp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, dp,
                                C.c_int32]
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_get_threads.restype = C.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def state_dim(model: int) -> int:
    return {QUAD2D: 6, ACKERMANN: 4, QUAD5: 5}.get(model, 3)


def make_params(cfg: dict) -> _Params:
    """Marshal a parameter dict (keys as in ``_Params``; ``lambda`` accepted
    for ``lam``) into the oracle's struct.  Missing arrays default to zero.
    ``grid`` is an ny x nx array of signed distances (the grid map), with
    ``grid_ox``, ``grid_oy``, ``grid_res``; the struct keeps a reference."""
    p = _Params()
    for name, ctype in _Params._fields_:
        key = "lambda" if name == "lam" else name
        if key not in cfg or name in ("grid", "grid_nx", "grid_ny"):
            continue
        val = cfg[key]
        if hasattr(ctype, "_length_"):
            arr = np.zeros(ctype._length_)
            v = np.asarray(val, dtype=np.float64).ravel()
            arr[: v.size] = v
            setattr(p, name, ctype(*arr))
        else:
            setattr(p, name, val)
    if "shape" in cfg:
        p.n_shape = int(np.asarray(cfg["shape"]).reshape(-1, 2).shape[0])
    if cfg.get("grid") is not None:
        g = np.ascontiguousarray(cfg["grid"], dtype=np.float32)
        if g.ndim != 2 or min(g.shape) < 2:
            raise ValueError("grid must be ny x nx with nx, ny >= 2")
        p._grid_ref = g
        p.grid = g.ctypes.data_as(C.POINTER(C.c_float))
        p.grid_ny, p.grid_nx = g.shape
    return p


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter under one 64-bit key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = C.POINTER(C.c_uint32)
    lib.orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p),
                          out.ctypes.data_as(u32p))
    return out


def uniform(r: int) -> float:
    return _load().orc_uniform(int(r) & 0xFFFFFFFF)


def noise(cfg: dict, S_e: float, k: int, t: int, it: int):
    """One NLN draw (Eq. 11) for sample k, step t, iteration it.
    Returns (du[2], z[4])."""
    lib = _load()
    p = make_params(cfg)
    du = np.zeros(2)
    z = np.zeros(4)
    lib.orc_noise(C.byref(p), S_e, k, t, it, _dp(du), _dp(z))
    return du, z


def noise_batch(cfg: dict, S_e: float, K: int, T: int, it: int):
    """K x T NLN draws; returns (du[K,T,2], z[K,T,4])."""
    lib = _load()
    p = make_params(cfg)
    du = np.zeros((K, T, 2))
    z = np.zeros((K, T, 4))
    lib.orc_noise_batch(C.byref(p), S_e, K, T, it, _dp(du), _dp(z))
    return du, z


def dynamics(cfg: dict, x, v) -> np.ndarray:
    lib = _load()
    p = make_params(cfg)
    n = state_dim(p.model)
    x = _f64(x)
    v = _f64(v)
    xn = np.zeros(n)
    lib.orc_dynamics(C.byref(p), _dp(x), _dp(v), _dp(xn))
    return xn


def grid_h(cfg: dict, px: float, py: float) -> float:
    """The grid map's h at world point (px, py) (bilinear, clamped)."""
    lib = _load()
    p = make_params(cfg)
    return lib.orc_grid_h(C.byref(p), px, py)


def bsum(cfg: dict, obstacles, x):
    """Fused barrier at state x: (sum 1/max(h, h_eps), collided, min h)."""
    lib = _load()
    p = make_params(cfg)
    ob = _f64(obstacles).reshape(-1, 3)
    ob = np.ascontiguousarray(ob)
    x = _f64(x)
    B = C.c_double()
    coll = C.c_int32()
    mh = C.c_double()
    lib.orc_bsum(C.byref(p), _dp(ob), ob.shape[0], _dp(x), C.byref(B),
                 C.byref(coll), C.byref(mh))
    return B.value, bool(coll.value), mh.value


def simulate(cfg: dict, x0, V) -> np.ndarray:
    lib = _load()
    p = make_params(cfg)
    n = state_dim(p.model)
    V = _f64(V).reshape(-1, 2)
    p.T = V.shape[0]
    X = np.zeros((p.T + 1, n))
    lib.orc_simulate(C.byref(p), _dp(_f64(x0)), _dp(V), _dp(X))
    return X


def weights(S, lam: float):
    """Eq. 4 weights.  Returns (w, rho, Z)."""
    lib = _load()
    S = _f64(S)
    w = np.zeros_like(S)
    Z = C.c_double()
    rho = lib.orc_weights(_dp(S), S.size, lam, _dp(w), C.byref(Z))
    return w, rho, Z.value


def sgf(y, window: int, order: int) -> np.ndarray:
    """Savitzky-Golay smoothing of each column of ``y`` (T, or T x m) along
    its first axis (Algorithm 1's SGF): at each t the degree-``order``
    least-squares polynomial through the window around t (the first or last
    ``window`` samples near the ends), evaluated at t."""
    lib = _load()
    y = _f64(y)
    Y = y.reshape(y.shape[0], -1)
    out = np.zeros_like(Y)
    T, m = Y.shape
    if not (window % 2 == 1 and 0 <= order < window <= T and order <= 6):
        raise ValueError("need an odd window, order < window <= T, order <= 6")
    for d in range(m):
        col = np.ascontiguousarray(Y[:, d])
        o = np.zeros(T)
        lib.orc_sgf(_dp(col), 1, T, window, order, _dp(o), 1)
        out[:, d] = o
    return out.reshape(y.shape)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


@dataclass
class Controller:
    """Oracle controller state carried between iterations (Algorithm 1)."""
    U: np.ndarray
    S_e: float
    beta: float = 0.0
    first: bool = True
    iter: int = 0


def new_controller(cfg: dict, u_init=None) -> Controller:
    T = int(cfg["T"])
    U = np.zeros((T, 2)) if u_init is None else _f64(u_init).reshape(T, 2).copy()
    mu = float(cfg.get("mu_coarse", 0.0))
    S_e = mu * np.log(np.e) if mu > 0 else 1.0
    return Controller(U=U, S_e=float(S_e))


def step(cfg: dict, obstacles, x0, xref, ctl: Controller,
         want_du: bool = False, want_sens: bool = True) -> dict:
    """One Algorithm 1 iteration; mutates ``ctl`` (shift, S_e, beta, iter).

    ``xref`` is (T+1) x n.  Returns costs, coll, minh, weights, Ustar, u0,
    CB_star, beta_used, beta_d, rho, Z, the post-step state, du_eff
    (K x T x 2) when ``want_du``, and per sample ``sens`` (the barrier
    cost's first-order change per unit of position error at every shape
    point) and ``reach`` (the rollout's largest distance from x0), with
    which the tests bound the cost error an FP32 rollout may make (both zero
    without ``want_sens``: the timed CPU baseline leaves them out)."""
    lib = _load()
    p = make_params(cfg)
    K, T, n = p.K, p.T, state_dim(p.model)
    ob = np.ascontiguousarray(_f64(obstacles).reshape(-1, 3))
    x0 = _f64(x0)
    xref = _f64(xref, (T + 1, n))
    U = np.ascontiguousarray(ctl.U, dtype=np.float64).reshape(T, 2).copy()
    st = _State(U=_dp(U), S_e=ctl.S_e, beta=ctl.beta, first=int(ctl.first),
                iter=ctl.iter)
    res = {
        "costs": np.zeros(K), "coll": np.zeros(K, dtype=np.uint8),
        "minh": np.zeros(K), "weights": np.zeros(K),
        "Ustar": np.zeros((T, 2)), "u0": np.zeros(2),
        "sens": np.zeros(K), "reach": np.zeros(K),
    }
    du = np.zeros((K, T, 2)) if want_du else None
    out = _Out(costs=_dp(res["costs"]),
               coll=res["coll"].ctypes.data_as(C.POINTER(C.c_uint8)),
               minh=_dp(res["minh"]), weights=_dp(res["weights"]),
               du_eff=_dp(du) if want_du else C.POINTER(C.c_double)(),
               Ustar=_dp(res["Ustar"]), u0=_dp(res["u0"]),
               sens=_dp(res["sens"]) if want_sens else C.POINTER(C.c_double)(),
               reach=_dp(res["reach"]) if want_sens else C.POINTER(C.c_double)())
    rc = lib.orc_step(C.byref(p), _dp(ob), ob.shape[0], _dp(x0), _dp(xref),
                      C.byref(st), C.byref(out))
    if rc == -2:
        raise ValueError("sgf_window must be 0 or odd and <= T, with sgf_order < "
                         "sgf_window and <= 6")
    if rc != 0:
        raise MemoryError("oracle step failed to allocate")
    res.update(CB_star=out.CB_star, beta_used=out.beta_used, beta_d=out.beta_d,
               rho=out.rho, Z=out.Z)
    if want_du:
        res["du_eff"] = du
    ctl.U = U
    ctl.S_e = st.S_e
    ctl.beta = st.beta
    ctl.first = bool(st.first)
    ctl.iter = int(st.iter)
    res["U_next"] = U.copy()
    res["S_e_next"] = ctl.S_e
    return res


def sample_costs(cfg: dict, obstacles, x0, xref, ctl: Controller, ks) -> dict:
    """Cost-to-go, collision flag, min h, barrier sensitivity and reach (as
    in ``step``) of the listed samples, from the state ``ctl`` (not
    modified)."""
    lib = _load()
    p = make_params(cfg)
    T, n = p.T, state_dim(p.model)
    ob = np.ascontiguousarray(_f64(obstacles).reshape(-1, 3))
    x0 = _f64(x0)
    xref = _f64(xref, (T + 1, n))
    U = np.ascontiguousarray(ctl.U, dtype=np.float64).reshape(T, 2).copy()
    st = _State(U=_dp(U), S_e=ctl.S_e, beta=ctl.beta, first=int(ctl.first), iter=ctl.iter)
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    S = np.zeros(ks.size)
    coll = np.zeros(ks.size, dtype=np.uint8)
    mh = np.zeros(ks.size)
    sens = np.zeros(ks.size)
    reach = np.zeros(ks.size)
    lib.orc_sample_costs(C.byref(p), _dp(ob), ob.shape[0], _dp(x0), _dp(xref), C.byref(st),
                         ks.ctypes.data_as(C.POINTER(C.c_int32)), ks.size, _dp(S),
                         coll.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(mh), _dp(sens),
                         _dp(reach))
    return dict(costs=S, coll=coll, minh=mh, sens=sens, reach=reach)
