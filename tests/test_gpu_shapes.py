"""Every compiled work shape of the band kernels against the FP64 oracle.

The autotuner (and so the benchmark) may pick any compiled shape: bands of
768 to 6144 nodes with register budgets of 6 or 7 CTAs per SM in 2D, boxes
of 512 nodes per plane over 8 planes with budgets of 3 to 6 CTAs per SM in
3D (the smaller budgets spill a little).  Each one must
meet the parity bounds on subdomains that it cuts into several bands or
boxes (ragged last band, transmission rows and columns inside the band
perimeter)."""
import numpy as np
import pytest

import oracle
from paper_2006_14602_gb300 import pma
from paper_2006_14602_gb300 import workloads as W
from paper_2006_14602_gb300.autotune import _count

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def counts():
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()
    return {"tile_2d": _count("tile_2d"), "tile_3d": _count("tile_3d")}


def _err(x, ref, prob):
    return np.abs(x - ref.x).max() / max(prob.hi[a] - prob.lo[a] for a in range(prob.dim))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_2d_shape(counts, prec):
    n = (331, 297, 1)
    prob = W.Problem(dim=2, n=n, monitor=W.random_bumps(np.random.default_rng(4), 2, 4),
                     parts=(2, 3, 1), overlap=6, dt=W.dt_for(n, 2), tol=0.0, max_steps=45,
                     precision=prec)
    ref = oracle.solve(prob)
    assert counts["tile_2d"] >= 7
    for t in range(counts["tile_2d"]):
        x, _, info = pma.solve(prob, want_psi=False, tile_2d=t)
        assert info.steps == ref.steps
        assert _err(x, ref, prob) <= (1e-11 if prec == "fp64" else 1e-5), t


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_3d_shape(counts, prec):
    n = (45, 39, 50)
    prob = W.Problem(dim=3, n=n, monitor=W.shell_monitor(), parts=(2, 2, 2), overlap=4,
                     dt=W.dt_for(n, 3, cfl=0.05), tol=0.0, max_steps=25, precision=prec)
    ref = oracle.solve(prob)
    assert counts["tile_3d"] >= 5
    for t in range(counts["tile_3d"]):
        x, _, info = pma.solve(prob, want_psi=False, tile_3d=t)
        assert info.steps == ref.steps
        assert _err(x, ref, prob) <= (1e-11 if prec == "fp64" else 1e-5), t
