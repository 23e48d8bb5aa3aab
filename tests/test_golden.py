"""Hand-derived worked examples under tests/golden/, run through the oracle
(to double precision) and through the CUDA library (to the FP32 path's
tolerance).  Each fixture's comments give the derivation and the equations
it follows; every applied control is pinned by u_min = u_max, so the
expected values do not depend on the random draws."""
import ast
import glob
import math
import operator
import os

import numpy as np
import pytest

from paper_2504_06437_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIXTURES = sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))

_OPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul,
        ast.Div: operator.truediv, ast.Pow: operator.pow}
_NAMES = {"e": math.e, "pi": math.pi}
_FUNCS = {"ln": math.log, "sqrt": math.sqrt}


def _eval(expr: str) -> float:
    """Arithmetic on numbers, e, pi, ln() and sqrt() only."""
    def ev(n):
        if isinstance(n, ast.Expression):
            return ev(n.body)
        if isinstance(n, ast.Constant) and isinstance(n.value, (int, float)):
            return float(n.value)
        if isinstance(n, ast.BinOp) and type(n.op) in _OPS:
            return _OPS[type(n.op)](ev(n.left), ev(n.right))
        if isinstance(n, ast.UnaryOp) and isinstance(n.op, ast.USub):
            return -ev(n.operand)
        if isinstance(n, ast.Name) and n.id in _NAMES:
            return _NAMES[n.id]
        if isinstance(n, ast.Call) and isinstance(n.func, ast.Name) and n.func.id in _FUNCS:
            return _FUNCS[n.func.id](*[ev(a) for a in n.args])
        raise ValueError(f"unsupported expression: {expr}")
    return ev(ast.parse(expr, mode="eval"))


def load_fixture(path: str) -> dict:
    out = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, val = (s.strip() for s in line.split("=", 1))
        vals = [_eval(v.strip()) for v in val.split(",")]
        out[key] = vals[0] if len(vals) == 1 else np.array(vals)
    return out


def problem(fx: dict):
    """Parameters, obstacles, x0, xref and initial sequence of a fixture."""
    model = int(fx["model"])
    K, T = int(fx["K"]), int(fx["T"])
    p = W.base_params(model, K=K, T=T, dt=fx["dt"], seed=11)
    for k in ("Q", "Qf", "gamma_ctrl", "C_coll", "R_B", "gamma_bas", "mu_coarse", "x_goal"):
        if k in fx:
            p[k] = fx[k]
    if "sigma" in fx:
        p["sigma"] = list(fx["sigma"])
    pin = list(np.atleast_1d(fx["pin"]))
    p["u_min"], p["u_max"] = pin, pin
    n = W.state_dim(model)
    ob = np.asarray(fx.get("obstacles", np.zeros((0, 3))), dtype=np.float64).reshape(-1, 3)
    x0 = np.asarray(fx["x0"], dtype=np.float64).reshape(n)
    xref = np.zeros((T + 1, n))
    U = (np.asarray(fx["u_init"], dtype=np.float64).reshape(T, 2) if "u_init" in fx
         else np.zeros((T, 2)))
    return p, ob, x0, xref, U


def expectations(fx: dict, step: int) -> dict:
    pre = f"step{step}."
    return {k[len(pre):]: v for k, v in fx.items() if k.startswith(pre)}


def test_fixtures_present():
    assert len(FIXTURES) >= 3


@pytest.mark.parametrize("path", FIXTURES, ids=os.path.basename)
def test_oracle_reproduces_hand_derived_values(orc, path):
    fx = load_fixture(path)
    p, ob, x0, xref, U = problem(fx)
    ctl = orc.new_controller(p, u_init=U)
    for s in range(1, int(fx["steps"]) + 1):
        r = orc.step(p, ob, x0, xref, ctl)
        for key, want in expectations(fx, s).items():
            got = r["u0"] if key == "u0" else (ctl.S_e if key == "S_e_next" else r[key])
            np.testing.assert_allclose(got, np.broadcast_to(want, np.shape(got)), rtol=1e-13,
                                       atol=1e-15, err_msg=f"{os.path.basename(path)} step {s} {key}")


@pytest.mark.gpu
@pytest.mark.parametrize("path", FIXTURES, ids=os.path.basename)
def test_cuda_path_reproduces_hand_derived_values(path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06437_gb300 import binding
    fx = load_fixture(path)
    p, ob, x0, xref, U = problem(fx)
    with binding.Controller(p, u_init=U) as g:
        g.set_obstacles(ob)
        for s in range(1, int(fx["steps"]) + 1):
            g.step(x0, xref)
            u0 = g.get_control()
            dbg = g.get_debug()
            for key, want in expectations(fx, s).items():
                got = u0 if key == "u0" else dbg[key]
                # FP32 rollout: 1e-4 relative on costs, 1e-5 on the rest
                tol = 1e-4 if key == "costs" else 1e-5
                np.testing.assert_allclose(got, np.broadcast_to(want, np.shape(got)), rtol=tol,
                                           atol=1e-6, err_msg=f"{os.path.basename(path)} step {s} {key}")
