"""The allocation-free step (mppi_step_static) against the context API.

Callers such as real-time control loops may not allocate device memory
once they run, so the library offers one step that keeps its scratch in a
fixed array inside the library.  This test calls it through the C ABI, twice
in a row on the same caller-owned state, and checks u0, the shifted sequence,
the per-sample costs, the exploration rate and the barrier state against
mppi_step / mppi_get_control on the same inputs.  Both run the same step
kernel in the same launch shape, so the results must agree bit for bit.  The
cases cover the smoothing form, an empty obstacle set (no obstacle copy),
costs left to the scratch array (d_costs NULL), and a full-size problem
(K 65536, T 100, 200 obstacles) whose 2048 tiles take the two-level merge.
The file sorts last so that a run stopping at the first failure has run
every other test before it."""
import ctypes as C

import numpy as np
import pytest

from paper_2504_06437_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06437_gb300 import binding
    lib = binding.load()
    vp = C.c_void_p
    lib.mppi_step_static.argtypes = [C.POINTER(binding.Params), vp, C.c_int32, vp, vp, vp, vp, vp,
                                     vp, vp]
    return torch, binding, lib


def _world(case):
    if case == "stress":
        return W.unicycle_stress(0), (0, 0)
    w = W.quad2d(3, K=1024, T=40)
    if case == "no_obstacles":
        w.obstacles = np.zeros((0, 3))
    return w, ((9, 3) if case == "smoothed" else (0, 0))


@pytest.mark.parametrize("case", ["plain", "smoothed", "no_obstacles", "costs_in_scratch", "stress"])
def test_step_static_matches_context_api_two_calls(case):
    torch, binding, lib = _lib()
    world, sgf = _world(case)
    p = dict(world.params, sgf_window=sgf[0], sgf_order=sgf[1])
    K, T = p["K"], p["T"]
    J = world.obstacles.shape[0]
    x = world.x_start.copy()
    xref = world.reference(x)

    # reference: the context API (default launch shape, as the static step
    # takes), two steps from the same measurement
    ref = []
    with binding.Controller(p) as g:
        g.set_obstacles(world.obstacles)
        for _ in range(2):
            g.step(x, xref)
            u0, U = g.get_control(want_U=True)
            st = g.get_state()
            ref.append((u0, U, g.get_debug()["costs"], st["S_e"], st["beta"], st["iter"]))

    dev = torch.device("cuda")
    d_obst = torch.tensor(world.obstacles.reshape(-1, 3), dtype=torch.float64, device=dev).contiguous()
    d_x0 = torch.tensor(x, dtype=torch.float64, device=dev)
    d_xref = torch.tensor(xref, dtype=torch.float64, device=dev).contiguous()
    d_U = torch.zeros((T, 2), dtype=torch.float64, device=dev)
    mu = p["mu_coarse"]
    d_ctl = torch.tensor([mu if mu > 0 else 1.0, 0.0, 1.0, 0.0, 0.0], dtype=torch.float64,
                         device=dev)
    d_u0 = torch.zeros(2, dtype=torch.float64, device=dev)
    d_costs = None if case == "costs_in_scratch" else torch.zeros(K, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    params = binding.make_params(p)
    for i in range(2):
        rc = lib.mppi_step_static(C.byref(params), d_obst.data_ptr() if J else None, J,
                                  d_x0.data_ptr(), d_xref.data_ptr(), d_U.data_ptr(),
                                  d_ctl.data_ptr(), d_u0.data_ptr(),
                                  None if d_costs is None else d_costs.data_ptr(), s.cuda_stream)
        assert rc == 0, lib.mppi_last_error().decode()
        s.synchronize()
        u0_r, U_r, costs_r, Se_r, beta_r, it_r = ref[i]
        ctl = d_ctl.cpu().numpy()
        assert ctl[4] == 0.0                       # status: no bounded wait expired
        assert ctl[2] == 0.0 and ctl[3] == i + 1 == it_r
        np.testing.assert_array_equal(d_u0.cpu().numpy(), u0_r)
        np.testing.assert_array_equal(d_U.cpu().numpy(), U_r)
        if d_costs is not None:
            np.testing.assert_array_equal(d_costs.cpu().numpy(), costs_r)
        assert ctl[0] == Se_r
        assert ctl[1] == beta_r


def test_step_static_rejects_oversize_problem():
    torch, binding, lib = _lib()
    p = W.base_params(W.UNICYCLE, K=1 << 21, T=256, dt=0.05, seed=0)
    p["x_goal"] = np.zeros(3)
    dev = torch.device("cuda")
    buf = torch.zeros(1024, dtype=torch.float64, device=dev)
    params = binding.make_params(p)
    ptr = buf.data_ptr()
    rc = lib.mppi_step_static(C.byref(params), None, 0, ptr, ptr, ptr, ptr, ptr, None, None)
    assert rc == binding.MPPI_EINVAL
    assert b"static scratch" in lib.mppi_last_error()
