"""Failure detection on the device without a GPU fault: the band kernel's
TMA staging wait is bounded.  The test hook announces more bytes to the
staging barrier than the copy delivers, so the wait runs out after about a
second; the kernel records the failure in the device error word and leaves,
the host turns it into PMA_ERR_TIMEOUT, and the GPU (and a new context)
keep working."""
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


def test_stalled_staging_wait_reports_timeout():
    p = W.small_case(2, 41, parts=(2, 2, 1), overlap=4, steps=24, precision="fp32")
    with pma.Context(0, window_steps=8, test_stall=1) as ctx:
        rid = ctx.submit(p)
        with pytest.raises(pma.PmaError) as e:
            ctx.run(4)
        assert e.value.status == pma.PMA_ERR_TIMEOUT
        # the error word was cleared: with the hook off the context runs on,
        # and the request retired with the timeout status
        ctx.set("test_stall", 0)
        ctx.run(1)
        x = np.empty((2, 41, 41))
        st, info = pma.pma_get_mesh(ctx.h, rid, x, None)
        assert st == pma.PMA_ERR_TIMEOUT and info.status == pma.PMA_ERR_TIMEOUT
    # the device is healthy: a new request solves and matches the oracle
    x, _, info = pma.solve(p, want_psi=False)
    ref = oracle.solve(p.replace(precision="fp64"))
    assert info.steps == ref.steps
    assert np.abs(x - ref.x).max() <= 1e-5


def test_stall_option_is_validated():
    with pma.Context(0) as ctx:
        with pytest.raises(pma.PmaError):
            ctx.set("test_stall", 2)
        ctx.set("test_stall", 0)
