"""The FP64 positivity check of a finished request (pma_check_mesh): min det
of the FD Hessian, min leading minor, min signed cell measure and count of
non-positive cells, against the oracle's quality measures of the same mesh."""
import numpy as np
import pytest

import oracle
from paper_2006_14602_gb300 import pma
from paper_2006_14602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()


def _check_request(prob):
    with pma.Context(0) as ctx:
        rid = ctx.submit(prob)
        ctx.run()
        st, out = pma.pma_check_mesh(ctx.h, rid)
        assert st == pma.PMA_OK, pma.pma_last_error()
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_check_matches_oracle_on_a_single_domain(dim):
    if dim == 2:
        prob = W.config1().replace(max_steps=500)
    else:
        prob = W.Problem(dim=3, n=(17, 15, 13), monitor=W.shell_monitor(),
                         dt=W.dt_for((17, 15, 13), 3, cfl=0.05), tol=0.0, max_steps=60,
                         precision="fp64")
    ref = oracle.solve(prob)
    q = oracle.quality(prob, ref.psi)
    out = _check_request(prob)
    assert out[0] > 0 and out[1] > 0 and out[2] > 0 and out[3] == 0
    assert abs(out[0] - q["min_det"]) <= 1e-9 * abs(q["min_det"])
    assert abs(out[2] - q["min_cell"]) <= 1e-9 * abs(q["min_cell"])


def test_check_on_decomposed_requests():
    """Decomposed requests: the cell measures of the combined (owner-takes)
    mesh equal the oracle's, and min det (each global node's det D_h^2 Psi
    from its owner's stencil, in FP64) equals the minimum of the oracle's
    owner-stencil determinants.  A request that tangled returns the last
    valid state: the tangling can sit in an overlap copy that the combined
    mesh does not use, so its combined mesh stays valid, as the oracle's."""
    prob = W.Problem(dim=2, n=(45, 37, 1), monitor=W.ring_monitor(), parts=(3, 2, 1), overlap=5,
                     dt=W.dt_for((45, 37, 1), 2), tol=0.0, max_steps=150, precision="fp64")
    bad = W.small_case(2, 25, parts=(2, 2, 1), overlap=4, steps=400).replace(
        dt=W.dt_for((25, 25, 1), 2, cfl=4.0))
    alt = prob.replace(alternating=1, exchange_every=3)
    for p in (prob, bad, alt):
        ref = oracle.solve(p, want_det=True)
        q = oracle.quality(p, ref.psi)
        out = _check_request(p)
        assert abs(out[2] - q["min_cell"]) <= 1e-9 * abs(q["min_cell"])
        assert (out[3] == 0) == (q["min_cell"] > 0)
        dmin = float(ref.det.min())
        assert abs(out[0] - dmin) <= 1e-9 * abs(dmin), (out[0], dmin)
