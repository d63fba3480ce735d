"""Continuous batching on the device: requests submitted while others are
running are admitted at window boundaries as memory allows, and every
result is bitwise the same as the request solved alone."""
import threading
import time

import numpy as np
import pytest

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


def _stream(n=14):
    reqs = [r for _, r in W.config5_stream(seed=5, count=n, rate_hz=200.0, max_steps=300,
                                           size2d=(33, 129), size3d=(17, 33))]
    reqs[3] = reqs[3].replace(precision="fp64")
    reqs[7] = reqs[7].replace(precision="fp64")
    return reqs


@pytest.mark.parametrize("resident", [0, 4])
def test_served_results_equal_alone(resident):
    reqs = _stream()
    alone = [pma.solve(r, want_psi=False, resident=resident) for r in reqs]
    with pma.Context(0, window_steps=16, resident=resident) as ctx:
        assert pma.pma_serve_start(ctx.h) == pma.PMA_OK
        ids = []

        def producer():
            for r in reqs:
                ids.append(ctx.submit(r))
                time.sleep(0.002)

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        for i in ids:
            st = pma.pma_wait(ctx.h, i, 60_000_000)
            # a random request may tangle; it must do so exactly as alone
            assert st in (pma.PMA_OK, pma.PMA_NOT_CONVERGED, pma.PMA_ERR_TANGLED), st
        assert pma.pma_serve_stop(ctx.h) == pma.PMA_OK
        for r, i, (xa, _, ia) in zip(reqs, ids, alone):
            x, _, info = ctx.mesh(r, i)
            assert info.status == ia.status and info.steps == ia.steps
            assert np.array_equal(x, xa)


def test_admission_waits_for_memory_budget():
    """A budget that holds one request at a time still serves all of them:
    a finished request keeps its memory until its mesh is fetched (which
    releases it), and the next queued one is admitted at the following
    window."""
    reqs = [W.small_case(2, 40, parts=(2, 2, 1), overlap=4, steps=80, precision="fp32")
            for _ in range(4)]
    alone = pma.solve(reqs[0], want_psi=False)
    # Four 22 x 22 subdomains (pitch 24), two FP32 buffers each, every buffer
    # rounded up to 256 bytes: 8 x 2304 = 18432 bytes per request.
    one = 8 * 2304
    with pma.Context(0, mem_budget_bytes=one + one // 2, window_steps=16) as ctx:
        ids = [ctx.submit(r) for r in reqs]
        st, (q, a, f) = pma.pma_counts(ctx.h)
        assert q == 4 and a == 0
        pending = list(zip(reqs, ids))
        windows = 0
        while pending:
            r, i = pending[0]
            st, done = pma.pma_poll(ctx.h, i)
            assert st == pma.PMA_OK
            if done:
                x, _, info = ctx.mesh(r, i)
                assert np.array_equal(x, alone[0])
                assert pma.pma_release(ctx.h, i) == pma.PMA_ERR_NOT_FOUND
                pending.pop(0)
                continue
            ctx.run(max_windows=1)
            st, (q, a, f) = pma.pma_counts(ctx.h)
            assert a <= 1
            windows += 1
            assert windows < 100


def test_oversized_request_is_rejected():
    with pma.Context(0, mem_budget_bytes=1 << 20) as ctx:
        big = W.small_case(2, 400, steps=1)
        with pytest.raises(pma.PmaError) as e:
            ctx.submit(big)
        assert e.value.status == pma.PMA_ERR_NOMEM


def test_wait_timeout_and_poll():
    prob = W.config1().replace(max_steps=20000)
    with pma.Context(0, window_steps=8) as ctx:
        assert pma.pma_serve_start(ctx.h) == pma.PMA_OK
        rid = ctx.submit(prob)
        st = pma.pma_wait(ctx.h, rid, 1)  # 1 microsecond: cannot be done yet
        assert st in (pma.PMA_ERR_TIMEOUT, pma.PMA_OK)
        assert pma.pma_wait(ctx.h, rid, 120_000_000) == pma.PMA_OK
        st, done = pma.pma_poll(ctx.h, rid)
        assert st == pma.PMA_OK and done == 1
        assert pma.pma_serve_stop(ctx.h) == pma.PMA_OK


def test_sweep_timing_and_launch_counters():
    """PMA_OPT_TIME_SWEEPS=k times the sweep launch of every k-th step: the
    timed launches are counted, their device time is positive and below the
    windows' time, and sweep and finish launches are counted apart."""
    prob = W.small_case(2, 40, parts=(2, 2, 1), overlap=4, steps=64, precision="fp32")
    with pma.Context(0, window_steps=16, time_sweeps=4) as ctx:
        ctx.submit(prob)
        ctx.run()
        _, s = pma.pma_get_stats(ctx.h)
    # INIT_V, INIT_THETA and 64 steps: 66 sweep launches in 5 windows of 16
    assert s.sweep_launches == s.windows * 16
    assert s.sweep_kernel_launches == s.windows * 4
    assert 0 < s.sweep_kernel_ms < s.window_ms
    assert s.other_launches >= s.windows * 16  # one finish per sweep, plus the combine
