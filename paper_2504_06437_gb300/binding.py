"""Thin ctypes binding over ``libdbasmppi.so`` (C ABI in ``include/dbasmppi.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no fallback; if the library is missing the import of
``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_LIB = os.path.join(_HERE, "libdbasmppi.so")
_SOURCES = ["csrc/dbasmppi.cu", "csrc/k_step_u.cu", "csrc/k_step_q.cu", "csrc/k_step_a.cu",
            "csrc/k_step_p.cu", "csrc/k_step_u_r80.cu", "csrc/k_step_q_r80.cu",
            "csrc/k_step_a_r80.cu", "csrc/k_step_p_r80.cu", "csrc/k_step_u_sgf.cu",
            "csrc/k_step_q_sgf.cu", "csrc/k_step_a_sgf.cu", "csrc/k_step_p_sgf.cu",
            "csrc/k_step_u_grid.cu", "csrc/k_step_q_grid.cu", "csrc/k_step_a_grid.cu",
            "csrc/k_step_p_grid.cu", "csrc/k_batch.cu", "csrc/k_batch_all.cu"]
_DEPS = _SOURCES + ["csrc/mppi_device.cuh", "csrc/mppi_tile.cuh", "csrc/kernels.cuh"]
HEADER = os.path.join(_ROOT, "include", "dbasmppi.h")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread"]

MPPI_OK, MPPI_EINVAL, MPPI_ENOMEM, MPPI_ECUDA, MPPI_ETIMEOUT, MPPI_ESTATE = 0, -1, -2, -3, -4, -5
UNICYCLE, QUAD2D, ACKERMANN, QUAD5 = 0, 1, 2, 3
NUM_MODELS = 4


def state_dim(model: int) -> int:
    return {QUAD2D: 6, ACKERMANN: 4, QUAD5: 5}.get(int(model), 3)
MAX_SHAPE = 8


class MppiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _stale() -> bool:
    if not os.path.exists(_LIB):
        return True
    t = os.path.getmtime(_LIB)
    deps = [os.path.join(_HERE, d) for d in _DEPS] + [HEADER]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library in-tree for sm_103a (nvcc cross-compiles
    without a GPU): each translation unit in parallel, then one shared link."""
    if not force and not _stale():
        return _LIB
    from concurrent.futures import ThreadPoolExecutor
    extra = os.environ.get("DBASMPPI_NVCC_EXTRA", "").split()
    objdir = os.path.join(_HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    tag = os.getpid()
    objs = [os.path.join(objdir, os.path.basename(src).replace(".cu", f".{tag}.o")) for src in _SOURCES]

    def compile_one(i):
        cmd = ["nvcc", *NVCC_FLAGS, *extra, "-c", "-o", objs[i], os.path.join(_HERE, _SOURCES[i])]
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)

    with ThreadPoolExecutor(len(_SOURCES)) as ex:
        list(ex.map(compile_one, range(len(_SOURCES))))
    tmp = _LIB + f".tmp{tag}"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs,
                    "-lpthread"], check=True)
    os.replace(tmp, _LIB)
    for o in objs:
        os.remove(o)
    return _LIB


class Params(C.Structure):
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
        ("shape", C.c_double * (2 * MAX_SHAPE)),
        ("seed", C.c_uint64),
        ("mass", C.c_double), ("inertia", C.c_double),
        ("arm", C.c_double), ("gravity", C.c_double),
        ("wheelbase", C.c_double),
        ("sgf_window", C.c_int32), ("sgf_order", C.c_int32),
    ]


class Tiling(C.Structure):
    _fields_ = [("samples_per_cta", C.c_int32), ("threads", C.c_int32),
                ("positions_per_thread", C.c_int32), ("chunk_steps", C.c_int32)]


class BatchPolicy(C.Structure):
    _fields_ = [("samples_per_cta", C.c_int32 * NUM_MODELS),
                ("positions_per_thread", C.c_int32 * NUM_MODELS)]


class ServerPolicy(C.Structure):
    _fields_ = [("small_ops_max", C.c_double), ("small_lanes", C.c_int32),
                ("shortest_first", C.c_int32), ("large_share", C.c_double),
                ("batch_ops_small", C.c_double), ("batch_ops_large", C.c_double),
                ("max_wait_s", C.c_double), ("device_queue", C.c_int32), ("reserved", C.c_int32)]


_lib = None
_dp = C.POINTER(C.c_double)


def load():
    """Load (building if needed) the library and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if _stale():
        build()
    lib = C.CDLL(_LIB)
    vp = C.c_void_p
    lib.mppi_create.argtypes = [C.POINTER(Params), _dp, C.POINTER(vp)]
    lib.mppi_create_tiled.argtypes = [C.POINTER(Params), _dp, C.POINTER(Tiling), C.POINTER(vp)]
    lib.mppi_set_obstacles.argtypes = [vp, _dp, C.c_int32]
    lib.mppi_set_grid.argtypes = [vp, C.POINTER(C.c_float), C.c_int32, C.c_int32, C.c_double,
                                  C.c_double, C.c_double]
    lib.mppi_step.argtypes = [vp, _dp, _dp, vp]
    lib.mppi_step_device.argtypes = [vp, vp, vp, vp]
    lib.mppi_get_control.argtypes = [vp, _dp, _dp]
    lib.mppi_get_debug.argtypes = [vp, _dp, C.POINTER(C.c_uint8), _dp, _dp, _dp]
    lib.mppi_io_bytes.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    lib.mppi_get_tiling.argtypes = [vp, C.POINTER(Tiling), C.POINTER(C.c_int32)]
    lib.mppi_get_kernel_regs.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.mppi_get_state.argtypes = [vp, _dp, _dp, _dp, C.POINTER(C.c_int32), C.POINTER(C.c_uint64)]
    lib.mppi_set_state.argtypes = [vp, _dp, C.c_double, C.c_double, C.c_int32, C.c_uint64]
    lib.mppi_destroy.argtypes = [vp]
    lib.mppi_debug_draws.argtypes = [C.POINTER(Params), C.c_double, C.c_uint64, C.c_int32,
                                     C.c_int32, C.POINTER(C.c_uint32), C.POINTER(C.c_float)]
    lib.mppi_debug_wait_probe.argtypes = [C.c_int64, C.c_int32]
    lib.mppi_autotune_grid.argtypes = [C.POINTER(Params), _dp, C.c_int32, C.POINTER(C.c_float),
                                       C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                       C.c_int32, C.POINTER(Tiling), C.POINTER(C.c_float)]
    lib.mppi_autotune.argtypes = [C.POINTER(Params), _dp, C.c_int32, C.c_int32,
                                  C.POINTER(Tiling), C.POINTER(C.c_float)]
    lib.mppi_autotune_flush.argtypes = [C.POINTER(Params), _dp, C.c_int32, C.POINTER(C.c_float),
                                        C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                        C.c_int32, C.c_uint64, C.POINTER(Tiling),
                                        C.POINTER(C.c_float)]
    lib.mppi_batch_create.argtypes = [C.c_int32, C.c_size_t, C.POINTER(vp)]
    lib.mppi_batch_add.argtypes = [vp, C.POINTER(Params), _dp, C.POINTER(Tiling), _dp, C.c_int32,
                                   C.POINTER(C.c_int32)]
    lib.mppi_batch_set_obstacles.argtypes = [vp, C.c_int32, _dp, C.c_int32]
    lib.mppi_batch_remove.argtypes = [vp, C.c_int32]
    lib.mppi_batch_step.argtypes = [vp, C.POINTER(C.c_int32), C.c_int32, _dp,
                                    C.POINTER(_dp), vp]
    lib.mppi_batch_get_controls.argtypes = [vp, _dp, C.c_int32]
    lib.mppi_batch_get_state.argtypes = [vp, C.c_int32, _dp, _dp, _dp]
    lib.mppi_batch_info.argtypes = [vp, C.c_int32, C.POINTER(Tiling), C.POINTER(C.c_uint64),
                                    C.POINTER(C.c_uint64)]
    lib.mppi_batch_set_graph.argtypes = [vp, C.c_int32]
    lib.mppi_batch_set_policy.argtypes = [vp, C.POINTER(BatchPolicy)]
    lib.mppi_batch_get_policy.argtypes = [vp, C.POINTER(BatchPolicy)]
    lib.mppi_batch_autotune.argtypes = [C.POINTER(Params), C.POINTER(_dp), C.POINTER(C.c_int32),
                                        C.c_int32, C.c_int32, C.c_size_t,
                                        C.POINTER(BatchPolicy), C.POINTER(C.c_float)]
    lib.mppi_batch_destroy.argtypes = [vp]
    lib.mppi_server_create.argtypes = [C.c_int32, C.c_size_t, C.c_int32, C.POINTER(vp)]
    lib.mppi_server_join.argtypes = [vp, C.POINTER(Params), _dp, _dp, C.c_int32,
                                     C.POINTER(C.c_int32)]
    lib.mppi_server_leave.argtypes = [vp, C.c_int32]
    lib.mppi_server_submit.argtypes = [vp, C.c_int32, _dp, _dp]
    lib.mppi_server_poll.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32), _dp, _dp, _dp,
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.mppi_server_poll_timed.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32), _dp, _dp, _dp, _dp,
                                           _dp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                           C.POINTER(C.c_int32)]
    lib.mppi_server_set_policy.argtypes = [vp, C.POINTER(ServerPolicy)]
    lib.mppi_server_get_policy.argtypes = [vp, C.POINTER(ServerPolicy), C.POINTER(C.c_int32)]
    lib.mppi_server_stats.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                      C.POINTER(C.c_int32), C.POINTER(C.c_uint64)]
    lib.mppi_server_destroy.argtypes = [vp]
    lib.mppi_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(rc: int):
    if rc != MPPI_OK:
        raise MppiError(rc, load().mppi_last_error().decode())


def make_params(cfg: dict) -> Params:
    p = Params()
    for name, ctype in Params._fields_:
        key = "lambda" if name == "lam" else name
        if key not in cfg:
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
    return p


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def debug_draws(cfg: dict, S_e: float, it: int, K: int, T: int):
    """Device generator output: (raw words [K,T,4] uint32, du [K,T,2] float32)."""
    p = make_params(cfg)
    raw = np.zeros((K, T, 4), dtype=np.uint32)
    du = np.zeros((K, T, 2), dtype=np.float32)
    _check(load().mppi_debug_draws(C.byref(p), float(S_e), int(it), int(K), int(T),
                                   raw.ctypes.data_as(C.POINTER(C.c_uint32)),
                                   du.ctypes.data_as(C.POINTER(C.c_float))))
    return raw, du


def autotune(cfg: dict, obstacles, iters: int = 10, flush_bytes: int = 0):
    """Fastest launch shape for this problem: (tiling dict, microseconds per step).
    A grid map in cfg (``grid``, ``grid_ox``, ``grid_oy``, ``grid_res``) is
    set on every candidate.  flush_bytes > 0 times each candidate step alone
    after a device write of that size (mppi_autotune_flush)."""
    p = make_params(cfg)
    ob = _f64(obstacles).reshape(-1, 3)
    t = Tiling()
    us = C.c_float()
    g = cfg.get("grid")
    gp, nx, ny, gox, goy, gres = None, 0, 0, 0.0, 0.0, 0.0
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float32)
        gp, nx, ny = g.ctypes.data_as(C.POINTER(C.c_float)), g.shape[1], g.shape[0]
        gox, goy, gres = float(cfg["grid_ox"]), float(cfg["grid_oy"]), float(cfg["grid_res"])
    _check(load().mppi_autotune_flush(C.byref(p), _ptr(ob) if ob.size else None, ob.shape[0], gp,
                                      nx, ny, gox, goy, gres, int(iters), int(flush_bytes),
                                      C.byref(t), C.byref(us)))
    return dict(samples_per_cta=t.samples_per_cta, threads=t.threads,
                positions_per_thread=t.positions_per_thread, chunk_steps=0), float(us.value)


class Controller:
    """One DBaS-Log-MPPI controller living on the GPU."""

    def __init__(self, cfg: dict, u_init=None, tiling: dict | None = None):
        lib = load()
        self.cfg = dict(cfg)
        self.params = make_params(cfg)
        self.K, self.T = int(self.params.K), int(self.params.T)
        self.n = state_dim(self.params.model)
        h = C.c_void_p()
        u = None if u_init is None else _f64(u_init).reshape(self.T, 2)
        self._u_init = u
        if tiling:
            t = Tiling(**{k: int(v) for k, v in tiling.items()})
            rc = lib.mppi_create_tiled(C.byref(self.params), _ptr(u) if u is not None else None,
                                       C.byref(t), C.byref(h))
        else:
            rc = lib.mppi_create(C.byref(self.params), _ptr(u) if u is not None else None, C.byref(h))
        _check(rc)
        self.h = h
        # per-controller argument buffers with their ctypes pointers made
        # once: numpy's pointer conversion costs microseconds per call, more
        # than the rest of a step's host work
        self._x0b = np.zeros(self.n)
        self._xrb = np.zeros((self.T + 1, self.n))
        self._u0b = np.zeros(2)
        self._Ub = np.zeros((self.T, 2))
        self._px0, self._pxr = _ptr(self._x0b), _ptr(self._xrb)
        self._pu0, self._pU = _ptr(self._u0b), _ptr(self._Ub)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().mppi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_obstacles(self, obstacles):
        ob = _f64(obstacles).reshape(-1, 3)
        _check(load().mppi_set_obstacles(self.h, _ptr(ob) if ob.size else None, ob.shape[0]))

    def set_grid(self, sdf, ox: float = 0.0, oy: float = 0.0, res: float = 1.0):
        """Set the grid map (ny x nx signed distances, sample (i, j) at
        (ox + i res, oy + j res)), or remove it with sdf=None."""
        if sdf is None:
            _check(load().mppi_set_grid(self.h, None, 0, 0, 0.0, 0.0, 0.0))
            return
        g = np.ascontiguousarray(sdf, dtype=np.float32)
        if g.ndim != 2:
            raise ValueError("grid must be a 2-D array (ny x nx)")
        _check(load().mppi_set_grid(self.h, g.ctypes.data_as(C.POINTER(C.c_float)), g.shape[1],
                                    g.shape[0], float(ox), float(oy), float(res)))

    def step(self, x0, xref=None, stream=None):
        self._x0b[:] = x0
        pxr = None
        if xref is not None:
            self._xrb[...] = np.asarray(xref, dtype=np.float64).reshape(self.T + 1, self.n)
            pxr = self._pxr
        _check(load().mppi_step(self.h, self._px0, pxr, _stream_ptr(stream)))

    def step_device(self, d_x0: int, d_xref: int, stream=None):
        _check(load().mppi_step_device(self.h, C.c_void_p(d_x0), C.c_void_p(d_xref),
                                       _stream_ptr(stream)))

    def get_control(self, want_U: bool = False):
        _check(load().mppi_get_control(self.h, self._pu0, self._pU if want_U else None))
        u0 = self._u0b.copy()
        return (u0, self._Ub.copy()) if want_U else u0

    def get_debug(self) -> dict:
        K, T = self.K, self.T
        costs = np.zeros(K)
        coll = np.zeros(K, dtype=np.uint8)
        w = np.zeros(K)
        Us = np.zeros((T, 2))
        sc = np.zeros(8)
        _check(load().mppi_get_debug(self.h, _ptr(costs), coll.ctypes.data_as(C.POINTER(C.c_uint8)),
                                     _ptr(w), _ptr(Us), _ptr(sc)))
        return dict(costs=costs, coll=coll, weights=w, Ustar=Us, rho=sc[0], Z=sc[1],
                    CB_star=sc[2], S_e_next=sc[3], beta_used=sc[4], beta_d=sc[5],
                    S_e_used=sc[6], iter=int(sc[7]))

    def tiling(self):
        t = Tiling()
        n = C.c_int32()
        _check(load().mppi_get_tiling(self.h, C.byref(t), C.byref(n)))
        return dict(samples_per_cta=t.samples_per_cta, threads=t.threads,
                    positions_per_thread=t.positions_per_thread, chunk_steps=t.chunk_steps,
                    n_ctas=n.value)

    def kernel_regs(self) -> int:
        """Register cap of the step kernel this controller launches (96 or 80)."""
        r = C.c_int32()
        _check(load().mppi_get_kernel_regs(self.h, C.byref(r)))
        return r.value

    def io_bytes(self):
        a, b = C.c_uint64(), C.c_uint64()
        _check(load().mppi_io_bytes(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def get_state(self) -> dict:
        U = np.zeros((self.T, 2))
        S_e, beta = C.c_double(), C.c_double()
        first, it = C.c_int32(), C.c_uint64()
        _check(load().mppi_get_state(self.h, _ptr(U), C.byref(S_e), C.byref(beta), C.byref(first),
                                     C.byref(it)))
        return dict(U=U, S_e=S_e.value, beta=beta.value, first=bool(first.value), iter=it.value)

    def set_state(self, U, S_e, beta, first, it):
        U = _f64(U).reshape(self.T, 2)
        _check(load().mppi_set_state(self.h, _ptr(U), float(S_e), float(beta), int(bool(first)), int(it)))


class Batch:
    """Many controllers stepped by one persistent launch (mppi_batch_*)."""

    def __init__(self, max_ctrl: int, pool_bytes: int):
        h = C.c_void_p()
        _check(load().mppi_batch_create(int(max_ctrl), int(pool_bytes), C.byref(h)))
        self.h = h
        self.info = {}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().mppi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def add(self, cfg: dict, obstacles=None, u_init=None, tiling: dict | None = None) -> int:
        p = make_params(cfg)
        T = int(p.T)
        u = None if u_init is None else _f64(u_init).reshape(T, 2)
        t = Tiling(**{k: int(v) for k, v in tiling.items()}) if tiling else None
        ob = _f64(obstacles if obstacles is not None else np.zeros((0, 3))).reshape(-1, 3)
        slot = C.c_int32()
        _check(load().mppi_batch_add(self.h, C.byref(p), _ptr(u) if u is not None else None,
                                     C.byref(t) if t is not None else None,
                                     _ptr(ob) if ob.size else None, ob.shape[0], C.byref(slot)))
        self.info[slot.value] = (T, state_dim(p.model), int(p.K))
        return slot.value

    def set_obstacles(self, slot: int, obstacles):
        ob = _f64(obstacles).reshape(-1, 3)
        _check(load().mppi_batch_set_obstacles(self.h, int(slot), _ptr(ob) if ob.size else None,
                                               ob.shape[0]))

    def remove(self, slot: int):
        _check(load().mppi_batch_remove(self.h, int(slot)))
        self.info.pop(slot, None)

    def step(self, slots, x0s, xrefs=None, stream=None):
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        n = slots.size
        X = np.zeros((n, 6))
        for i, x in enumerate(x0s):
            x = np.asarray(x, dtype=np.float64).ravel()
            X[i, : x.size] = x
        self._keep = []
        ptrs = None
        if xrefs is not None:
            ptrs = (_dp * n)()
            for i, r in enumerate(xrefs):
                if r is None:
                    ptrs[i] = _dp()
                else:
                    a = _f64(r)
                    self._keep.append(a)
                    ptrs[i] = _ptr(a)
        self._keep.append(X)
        _check(load().mppi_batch_step(self.h, slots.ctypes.data_as(C.POINTER(C.c_int32)), n,
                                      _ptr(X), ptrs, _stream_ptr(stream)))
        self._n = n

    def controls(self) -> np.ndarray:
        u = np.zeros((self._n, 2))
        _check(load().mppi_batch_get_controls(self.h, _ptr(u), self._n))
        return u

    def state(self, slot: int) -> dict:
        T, n, K = self.info[slot]
        U = np.zeros((T, 2))
        costs = np.zeros(K)
        sc = np.zeros(8)
        _check(load().mppi_batch_get_state(self.h, int(slot), _ptr(U), _ptr(costs), _ptr(sc)))
        return dict(U=U, costs=costs, rho=sc[0], Z=sc[1], CB_star=sc[2], S_e=sc[3],
                    beta_used=sc[4], beta_d=sc[5], S_e_used=sc[6], iter=int(sc[7]))

    def slot_info(self, slot: int = -1) -> dict:
        t = Tiling()
        b = C.c_uint64()
        f = C.c_uint64()
        _check(load().mppi_batch_info(self.h, int(slot), C.byref(t), C.byref(b), C.byref(f)))
        return dict(samples_per_cta=t.samples_per_cta, threads=t.threads,
                    positions_per_thread=t.positions_per_thread, bytes=b.value, pool_free=f.value)

    def set_graph(self, enable: bool):
        _check(load().mppi_batch_set_graph(self.h, int(bool(enable))))

    def set_policy(self, policy: dict):
        """Launch shape for later adds without an explicit tiling: dict with
        per-model lists samples_per_cta and positions_per_thread."""
        _check(load().mppi_batch_set_policy(self.h, C.byref(_policy(policy))))

    def get_policy(self) -> dict:
        pol = BatchPolicy()
        _check(load().mppi_batch_get_policy(self.h, C.byref(pol)))
        return _policy_dict(pol)


def _policy(d: dict) -> BatchPolicy:
    """Per-model lists; models past the end of a shorter list take the
    library's defaults (32 samples per CTA, points per thread chosen)."""
    pol = BatchPolicy()
    S, NP = list(d["samples_per_cta"]), list(d["positions_per_thread"])
    for m in range(NUM_MODELS):
        pol.samples_per_cta[m] = int(S[m]) if m < len(S) else 32
        pol.positions_per_thread[m] = int(NP[m]) if m < len(NP) else 0
    return pol


def _policy_dict(pol: BatchPolicy) -> dict:
    return dict(samples_per_cta=[pol.samples_per_cta[m] for m in range(NUM_MODELS)],
                positions_per_thread=[pol.positions_per_thread[m] for m in range(NUM_MODELS)])


def batch_autotune(cfgs, obstacles, iters: int = 3, pool_bytes: int = 2 << 30):
    """Fastest batch policy for these controllers: (policy dict, ms per batched step)."""
    n = len(cfgs)
    ps = (Params * n)(*[make_params(c) for c in cfgs])
    obs = [_f64(o).reshape(-1, 3) for o in obstacles]
    ptrs = (_dp * n)(*[_ptr(o) if o.size else None for o in obs])
    Js = (C.c_int32 * n)(*[o.shape[0] for o in obs])
    pol = BatchPolicy()
    ms = C.c_float()
    _check(load().mppi_batch_autotune(ps, ptrs, Js, n, int(iters), int(pool_bytes), C.byref(pol),
                                      C.byref(ms)))
    return _policy_dict(pol), float(ms.value)


class Server:
    """Continuous-batching serving runtime (mppi_server_*)."""

    def __init__(self, max_robots: int, pool_bytes: int, lanes: int = 2):
        h = C.c_void_p()
        _check(load().mppi_server_create(int(max_robots), int(pool_bytes), int(lanes), C.byref(h)))
        self.h = h
        self.dims = {}
        self._buf = 4096
        self._r = np.zeros(self._buf, dtype=np.int32)
        self._u = np.zeros((self._buf, 2))
        self._x = np.zeros((self._buf, 6))
        self._l = np.zeros(self._buf)
        self._q = np.zeros(self._buf)
        self._d = np.zeros(self._buf)
        self._c = np.zeros(self._buf, dtype=np.int32)
        self._s = np.zeros(self._buf, dtype=np.int32)
        self.lanes = int(lanes)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().mppi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def join(self, cfg: dict, obstacles, u_init=None):
        """Robot id, or None when admission is refused for lack of memory."""
        p = make_params(cfg)
        ob = _f64(obstacles).reshape(-1, 3)
        u = None if u_init is None else _f64(u_init).reshape(int(p.T), 2)
        r = C.c_int32()
        rc = load().mppi_server_join(self.h, C.byref(p), _ptr(u) if u is not None else None,
                                     _ptr(ob) if ob.size else None, ob.shape[0], C.byref(r))
        if rc == MPPI_ENOMEM:
            return None
        _check(rc)
        self.dims[r.value] = (int(p.T), state_dim(p.model))
        return r.value

    def leave(self, robot: int):
        _check(load().mppi_server_leave(self.h, int(robot)))
        self.dims.pop(robot, None)

    def submit(self, robot: int, x0, xref=None):
        x0 = _f64(x0)
        xr = None if xref is None else _f64(xref)
        _check(load().mppi_server_submit(self.h, int(robot), _ptr(x0),
                                         _ptr(xr) if xr is not None else None))

    def poll(self):
        """Completed requests: list of (robot, u0, predicted x1, latency s, status)."""
        n = C.c_int32()
        _check(load().mppi_server_poll(self.h, self._buf, self._r.ctypes.data_as(C.POINTER(C.c_int32)),
                                       _ptr(self._u), _ptr(self._x), _ptr(self._l),
                                       self._s.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)))
        k = n.value
        return [(int(self._r[i]), self._u[i].copy(), self._x[i].copy(), float(self._l[i]),
                 int(self._s[i])) for i in range(k)]

    def poll_timed(self):
        """Completed requests as dicts: robot, u0, x1, latency, queue and
        device seconds, size class (0 small or the only class, 1 large),
        status."""
        n = C.c_int32()
        i32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        _check(load().mppi_server_poll_timed(self.h, self._buf, i32(self._r), _ptr(self._u),
                                             _ptr(self._x), _ptr(self._l), _ptr(self._q),
                                             _ptr(self._d), i32(self._c), i32(self._s),
                                             C.byref(n)))
        return [dict(robot=int(self._r[i]), u0=self._u[i].copy(), x1=self._x[i].copy(),
                     latency=float(self._l[i]), queue=float(self._q[i]), device=float(self._d[i]),
                     size_class=int(self._c[i]), status=int(self._s[i])) for i in range(n.value)]

    def set_policy(self, small_ops_max: float, small_lanes: int = 1, large_share: float = 0.75,
                   batch_ops_small: float = 0.0, batch_ops_large: float = 0.0,
                   shortest_first: bool = False, max_wait_s: float = 0.0,
                   device_queue: bool = False):
        pol = ServerPolicy(float(small_ops_max), int(small_lanes), int(bool(shortest_first)),
                           float(large_share), float(batch_ops_small), float(batch_ops_large),
                           float(max_wait_s), int(bool(device_queue)), 0)
        _check(load().mppi_server_set_policy(self.h, C.byref(pol)))

    def get_policy(self) -> dict:
        pol = ServerPolicy()
        cls = (C.c_int32 * self.lanes)()
        _check(load().mppi_server_get_policy(self.h, C.byref(pol), cls))
        return dict(small_ops_max=pol.small_ops_max, small_lanes=pol.small_lanes,
                    shortest_first=bool(pol.shortest_first), large_share=pol.large_share,
                    batch_ops_small=pol.batch_ops_small, batch_ops_large=pol.batch_ops_large,
                    max_wait_s=pol.max_wait_s, device_queue=bool(pol.device_queue),
                    lane_classes=list(cls))

    def stats(self) -> dict:
        b, r, f = C.c_uint64(), C.c_uint64(), C.c_uint64()
        q = C.c_int32()
        _check(load().mppi_server_stats(self.h, C.byref(b), C.byref(r), C.byref(q), C.byref(f)))
        return dict(batches=b.value, requests=r.value, pending=q.value, pool_free=f.value)
