"""The allocation-free step (mppi_step_static) against the context API.

Callers such as real-time control loops may not allocate device memory
once they run, so the library offers one step that keeps its scratch in a
fixed array inside the library.  This test calls it through the C ABI, twice
in a row on the same caller-owned state, and checks u0, the shifted sequence,
the per-sample costs and the exploration rate against mppi_step /
mppi_get_control on the same inputs, within the parity tolerances used by the
other GPU tests.  The file sorts last so that a run stopping at the first
failure has run every other test before it."""
import ctypes as C

import numpy as np
import pytest

from paper_2504_06437_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U_ATOL = 1e-5
COST_RTOL = 1e-4


@pytest.mark.parametrize("sgf", [(0, 0), (9, 3)])
def test_step_static_matches_context_api_two_calls(sgf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06437_gb300 import binding
    lib = binding.load()
    vp = C.c_void_p
    lib.mppi_step_static.argtypes = [C.POINTER(binding.Params), vp, C.c_int32, vp, vp, vp, vp, vp,
                                     vp, vp]

    world = W.quad2d(3, K=1024, T=40)
    p = dict(world.params, sgf_window=sgf[0], sgf_order=sgf[1])
    K, T, n = p["K"], p["T"], world.n
    x = world.x_start.copy()
    xref = world.reference(x)

    # reference: the context API, two steps from the same measurement
    ref = []
    with binding.Controller(p) as g:
        g.set_obstacles(world.obstacles)
        for _ in range(2):
            g.step(x, xref)
            u0, U = g.get_control(want_U=True)
            st = g.get_state()
            ref.append((u0, U, g.get_debug()["costs"], st["S_e"], st["beta"]))

    dev = torch.device("cuda")
    d_obst = torch.tensor(world.obstacles, dtype=torch.float64, device=dev).contiguous()
    d_x0 = torch.tensor(x, dtype=torch.float64, device=dev)
    d_xref = torch.tensor(xref, dtype=torch.float64, device=dev).contiguous()
    d_U = torch.zeros((T, 2), dtype=torch.float64, device=dev)
    mu = p["mu_coarse"]
    d_ctl = torch.tensor([mu if mu > 0 else 1.0, 0.0, 1.0, 0.0, 0.0], dtype=torch.float64,
                         device=dev)
    d_u0 = torch.zeros(2, dtype=torch.float64, device=dev)
    d_costs = torch.zeros(K, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    params = binding.make_params(p)
    for i in range(2):
        rc = lib.mppi_step_static(C.byref(params), d_obst.data_ptr(), world.obstacles.shape[0],
                                  d_x0.data_ptr(), d_xref.data_ptr(), d_U.data_ptr(),
                                  d_ctl.data_ptr(), d_u0.data_ptr(), d_costs.data_ptr(),
                                  s.cuda_stream)
        assert rc == 0, lib.mppi_last_error().decode()
        s.synchronize()
        u0_r, U_r, costs_r, Se_r, beta_r = ref[i]
        ctl = d_ctl.cpu().numpy()
        assert ctl[4] == 0.0
        assert ctl[2] == 0.0 and ctl[3] == i + 1
        np.testing.assert_allclose(d_u0.cpu().numpy(), u0_r, rtol=0, atol=U_ATOL)
        np.testing.assert_allclose(d_U.cpu().numpy(), U_r, rtol=0, atol=U_ATOL)
        c = d_costs.cpu().numpy()
        assert np.max(np.abs(c - costs_r) / np.maximum(np.abs(costs_r), 1.0)) <= COST_RTOL
        assert ctl[0] == pytest.approx(Se_r, rel=1e-6)
        assert ctl[1] == pytest.approx(beta_r, rel=1e-6, abs=1e-9)


def test_step_static_rejects_oversize_problem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06437_gb300 import binding
    lib = binding.load()
    vp = C.c_void_p
    lib.mppi_step_static.argtypes = [C.POINTER(binding.Params), vp, C.c_int32, vp, vp, vp, vp, vp,
                                     vp, vp]
    p = W.base_params(W.UNICYCLE, K=1 << 21, T=256, dt=0.05, seed=0)
    p["x_goal"] = np.zeros(3)
    dev = torch.device("cuda")
    buf = torch.zeros(1024, dtype=torch.float64, device=dev)
    params = binding.make_params(p)
    ptr = buf.data_ptr()
    rc = lib.mppi_step_static(C.byref(params), None, 0, ptr, ptr, ptr, ptr, ptr, None, None)
    assert rc == binding.MPPI_EINVAL
    assert b"static scratch" in lib.mppi_last_error()
