"""The allocation-free solve (pma_solve_static) against the allocating path.

Some callers cannot allocate device memory when they need a mesh: their host
application reserved the whole device for its own pool, a framework's caching
allocator owns every byte, or the calling code must not risk the device-wide
synchronisation that an allocation or a free can cause.  pma_solve_static
serves them from a fixed scratch area inside the library.  These tests call
it through the C ABI twice in a row (the scratch keeps the previous call's
contents) and compare each result with the ordinary context path and with
the FP64 oracle, within the tolerances the other parity tests use.  The file is named to be collected
last, and it passes alone in a fresh process as well as after the suite.
"""
import numpy as np
import pytest

import oracle
from paper_2006_14602_gb300 import pma
from paper_2006_14602_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-5}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()
    return torch


CASES = {
    "2d_dd_fp64": W.Problem(dim=2, n=(45, 37, 1), monitor=W.ring_monitor(), parts=(3, 2, 1),
                            overlap=5, dt=W.dt_for((45, 37, 1), 2), tol=0.0, max_steps=150,
                            precision="fp64"),
    "2d_dd_fp32": W.Problem(dim=2, n=(97, 65, 1), monitor=W.sine_monitor(), parts=(4, 3, 1),
                            overlap=8, dt=W.dt_for((97, 65, 1), 2), tol=0.0, max_steps=120,
                            precision="fp32"),
    "2d_converging": W.config1().replace(max_steps=4000),
    "2d_alternating": W.Problem(dim=2, n=(40, 33, 1), monitor=W.ring_monitor(), parts=(2, 2, 1),
                                overlap=2, alternating=1, dt=W.dt_for((40, 33, 1), 2), tol=0.0,
                                max_steps=100, precision="fp64"),
    "2d_exchange3_fp32": W.Problem(dim=2, n=(50, 44, 1), monitor=W.ring_monitor(), parts=(2, 3, 1),
                                   overlap=4, exchange_every=3, dt=W.dt_for((50, 44, 1), 2),
                                   tol=0.0, max_steps=90, precision="fp32"),
    "3d_dd_fp64": W.Problem(dim=3, n=(19, 17, 15), monitor=W.shell_monitor(), parts=(2, 2, 2),
                            overlap=4, dt=W.dt_for((19, 17, 15), 3, cfl=0.05), tol=0.0,
                            max_steps=60, precision="fp64"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_static_solve_matches_allocating_path_twice(torch_cuda, name):
    torch = torch_cuda
    prob = CASES[name]
    ref_x, _, ref_info = pma.solve(prob, want_psi=False)
    exact = oracle.solve(prob.replace(precision="fp64"))
    g, m, d, p = pma.to_structs(prob)
    out = torch.empty(ref_x.size, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        st, info = pma.pma_solve_static(g, m, d, p, 0, out.data_ptr(), 0)
        assert st == ref_info.status, (st, pma.pma_last_error())
        assert info.steps == ref_info.steps == exact.steps
        x = out.cpu().numpy().reshape(ref_x.shape)
        assert np.abs(x - ref_x).max() <= TOL[prob.precision]
        assert np.abs(x - exact.x).max() <= TOL[prob.precision]


def test_static_solve_warm_start_on_device(torch_cuda):
    torch = torch_cuda
    prob = W.config1().replace(max_steps=200)
    first_x, first_psi, _ = pma.solve(prob, want_psi=True)
    ref_x, _, ref_info = pma.solve(prob, psi0=first_psi, want_psi=False)
    g, m, d, p = pma.to_structs(prob)
    psi0 = torch.from_numpy(np.ascontiguousarray(first_psi)).to("cuda")
    out = torch.empty(ref_x.size, dtype=torch.float64, device="cuda")
    for _ in range(2):
        st, info = pma.pma_solve_static(g, m, d, p, psi0.data_ptr(), out.data_ptr(), 0)
        assert st == ref_info.status and info.steps == ref_info.steps
        x = out.cpu().numpy().reshape(ref_x.shape)
        assert np.abs(x - ref_x).max() <= TOL["fp64"]


def test_static_solve_rejects_requests_beyond_the_scratch(torch_cuda):
    torch = torch_cuda
    big = W.Problem(dim=2, n=(3000, 3000, 1), monitor=W.ring_monitor(), dt=1e-8, tol=0.0,
                    max_steps=1, precision="fp32")
    g, m, d, p = pma.to_structs(big)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    st, _ = pma.pma_solve_static(g, m, d, p, 0, out.data_ptr(), 0)
    assert st == pma.PMA_ERR_NOMEM
    assert "scratch" in pma.pma_last_error()
