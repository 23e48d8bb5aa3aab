"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/dbasmppi.h declares, matches the binding's struct layout, and
rejects bad arguments before touching the GPU.  No GPU needed."""
import ctypes as C
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2504_06437_gb300 import binding, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mppi_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    binding.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mppi_create", "mppi_set_obstacles", "mppi_step", "mppi_get_control",
                     "mppi_destroy", "mppi_get_debug"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_header():
    """Compile a C probe against the header and compare sizeof/offsetof with
    the ctypes mirror."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc unavailable")
    fields = [f for f, _ in binding.Params._fields_]
    cname = {"lam": "lambda"}
    body = "\n".join(f'  printf("%zu\\n", offsetof(mppi_params, {cname.get(f, f)}));' for f in fields)
    prog = ("#include <stdio.h>\n#include <stddef.h>\n#include \"dbasmppi.h\"\nint main(void){\n"
            f'  printf("%zu\\n", sizeof(mppi_params));\n{body}\n'
            '  printf("%zu\\n", sizeof(mppi_tiling));\n  return 0;\n}\n')
    d = tempfile.mkdtemp()
    try:
        src, exe = os.path.join(d, "probe.c"), os.path.join(d, "probe")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    finally:
        shutil.rmtree(d, ignore_errors=True)
    assert out[0] == C.sizeof(binding.Params)
    for f, off in zip(fields, out[1:-1]):
        assert getattr(binding.Params, f).offset == off, f
    assert out[-1] == C.sizeof(binding.Tiling)


def test_server_policy_layout_matches_header():
    """The serving policy struct: sizeof/offsetof against the ctypes mirror."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc unavailable")
    fields = [f for f, _ in binding.ServerPolicy._fields_]
    body = "\n".join(f'  printf("%zu\\n", offsetof(mppi_server_policy, {f}));' for f in fields)
    prog = ("#include <stdio.h>\n#include <stddef.h>\n#include \"dbasmppi.h\"\nint main(void){\n"
            f'  printf("%zu\\n", sizeof(mppi_server_policy));\n{body}\n  return 0;\n}}\n')
    d = tempfile.mkdtemp()
    try:
        src, exe = os.path.join(d, "probe.c"), os.path.join(d, "probe")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    finally:
        shutil.rmtree(d, ignore_errors=True)
    assert out[0] == C.sizeof(binding.ServerPolicy)
    for f, off in zip(fields, out[1:]):
        assert getattr(binding.ServerPolicy, f).offset == off, f


def _bad(cfg_over):
    p = W.base_params(W.UNICYCLE, K=64, T=10, dt=0.05, seed=0)
    p.update(x_goal=np.zeros(3))
    p.update(cfg_over)
    return p


@pytest.mark.parametrize("over", [
    dict(K=0), dict(T=0), dict(T=100000), dict(model=7), {"lambda": 0.0}, {"lambda": -1.0},
    dict(gamma_bas=1.0), dict(gamma_bas=0.0), dict(h_eps=0.0), dict(dt=0.0),
    dict(sigma=[1.0, 0.5, 0.2, 1.0]), dict(sigma=[-1.0, 0.0, 0.0, 1.0]),
    dict(sigma=[0.0, 0.0, 0.0, 0.0]), dict(u_min=[1.0, 0.0], u_max=[0.0, 1.0]),
    dict(dt=float("nan")), dict(ln_sigma=-0.1), dict(n_shape=9), dict(n_shape=0),
    # Savitzky-Golay smoothing: even, too wide for T = 10, order >= window, order > 6
    dict(sgf_window=4, sgf_order=1), dict(sgf_window=11, sgf_order=2),
    dict(sgf_window=5, sgf_order=5), dict(sgf_window=9, sgf_order=7),
    dict(sgf_window=-3, sgf_order=0), dict(sgf_window=1, sgf_order=0),
])
def test_create_rejects_bad_params_without_gpu(lib, over):
    p = binding.make_params(_bad(over))
    if "n_shape" in over:
        p.n_shape = over["n_shape"]
    h = C.c_void_p()
    rc = lib.mppi_create(C.byref(p), None, C.byref(h))
    assert rc == binding.MPPI_EINVAL
    assert lib.mppi_last_error()
    assert not h.value


@pytest.mark.parametrize("nx,ny,res,value", [(1, 5, 0.1, 0.0), (5, 1, 0.1, 0.0), (4, 4, 0.0, 0.0),
                                             (4, 4, -0.5, 0.0), (4, 4, float("inf"), 0.0),
                                             (4, 4, 0.1, float("nan")), (70000, 2, 0.1, 0.0)])
def test_grid_rejected_without_gpu(lib, nx, ny, res, value):
    """The grid map's checks (sides, cell size, finite samples) run before
    any CUDA call: mppi_autotune_grid refuses a bad map on a host without a
    GPU."""
    p = binding.make_params(_bad({}))
    g = np.full((ny, nx), value, dtype=np.float32)
    t = binding.Tiling()
    us = C.c_float()
    rc = lib.mppi_autotune_grid(C.byref(p), None, 0, g.ctypes.data_as(C.POINTER(C.c_float)), nx, ny,
                                0.0, 0.0, res, 1, C.byref(t), C.byref(us))
    assert rc == binding.MPPI_EINVAL
    assert b"grid" in lib.mppi_last_error()


def test_autotune_flush_bound_without_gpu(lib):
    """mppi_autotune_flush refuses a flush write above 4 GiB before any CUDA
    call."""
    p = binding.make_params(_bad({}))
    t = binding.Tiling()
    us = C.c_float()
    rc = lib.mppi_autotune_flush(C.byref(p), None, 0, None, 0, 0, 0.0, 0.0, 0.0, 1, 5 << 30,
                                 C.byref(t), C.byref(us))
    assert rc == binding.MPPI_EINVAL
    assert b"flush" in lib.mppi_last_error()


def test_null_handles(lib):
    assert lib.mppi_destroy(None) == binding.MPPI_OK
    assert lib.mppi_step(None, None, None, None) == binding.MPPI_ESTATE
    assert lib.mppi_get_control(None, None, None) == binding.MPPI_ESTATE
    assert lib.mppi_set_obstacles(None, None, 0) == binding.MPPI_ESTATE
    assert lib.mppi_set_grid(None, None, 0, 0, 0.0, 0.0, 0.0) == binding.MPPI_ESTATE
