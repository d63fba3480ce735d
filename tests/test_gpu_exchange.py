"""Interface data frozen over K steps (exchange_every) on the device, against
the FP64 oracle.

Sect. 3 integrates every subdomain over a pseudo-time interval with its
neighbours' data of the interval's start; with forward Euler that is an
exchange of the transmission values every K steps and frozen Dirichlet data
in between.  Node positions must match the oracle within 1e-11 (FP64) and
1e-5 (FP32) of the domain size after the same steps, in both transmission
forms, in 2D and 3D, with window lengths that are not multiples of K.
"""
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


def _err(x, ref, prob):
    return np.abs(x - ref.x).max() / max(prob.hi[a] - prob.lo[a] for a in range(prob.dim))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("K", [2, 8])
@pytest.mark.parametrize("alt", [0, 1])
def test_exchange_every_2d(prec, K, alt):
    n = (57, 49, 1)
    prob = W.Problem(dim=2, n=n, monitor=W.ring_monitor(), parts=(3, 2, 1), overlap=4,
                     alternating=alt, exchange_every=K, dt=W.dt_for(n, 2), tol=0.0,
                     max_steps=203, precision=prec)
    ref = oracle.solve(prob)
    x, _, info = pma.solve(prob, want_psi=False, window_steps=12)
    assert info.steps == ref.steps == 203
    assert _err(x, ref, prob) <= (1e-11 if prec == "fp64" else 1e-5)
    # the frozen data matter: K differs from one exchange per step
    ref1 = oracle.solve(prob.replace(exchange_every=1))
    assert np.abs(ref1.x - ref.x).max() > 1e-7


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("K,alt", [(3, 0), (4, 1)])
def test_exchange_every_3d(prec, K, alt):
    n = (23, 19, 21)
    prob = W.Problem(dim=3, n=n, monitor=W.shell_monitor(), parts=(2, 2, 2), overlap=4,
                     alternating=alt, exchange_every=K, dt=W.dt_for(n, 3, cfl=0.05), tol=0.0,
                     max_steps=61, precision=prec)
    ref = oracle.solve(prob)
    x, _, info = pma.solve(prob, want_psi=False, window_steps=16)
    assert info.steps == ref.steps
    assert _err(x, ref, prob) <= (1e-11 if prec == "fp64" else 1e-5)


def test_exchange_every_stops_like_the_oracle():
    """Converged runs: the stop test sees the frozen-data residual; step
    count and status equal the oracle's, and the mesh is the single-domain
    steady state."""
    prob = W.Problem(dim=2, n=(33, 33, 1), monitor=W.ring_monitor(), parts=(2, 2, 1),
                     overlap=4, exchange_every=4, check_every=4, dt=1e-4, tol=1e-7,
                     max_steps=20000)
    ref = oracle.solve(prob)
    assert ref.status == "ok"
    x, _, info = pma.solve(prob, want_psi=False)
    assert info.steps == ref.steps and pma.STATUS_NAMES[info.status] == "ok"
    assert _err(x, ref, prob) <= 1e-11


def test_exchange_every_one_is_bitwise_the_default():
    prob = W.small_case(2, 41, parts=(2, 2, 1), overlap=4, steps=80)
    a, _, _ = pma.solve(prob, want_psi=False)
    b, _, _ = pma.solve(prob.replace(exchange_every=1), want_psi=False)
    np.testing.assert_array_equal(a, b)


def test_exchange_every_per_subdomain_launches_and_mix():
    """The plain one-launch-per-subdomain path gives the same result, and a
    frozen-data request is bitwise the same alone and in a mixed batch."""
    n = (45, 40, 1)
    prob = W.Problem(dim=2, n=n, monitor=W.sine_monitor(), parts=(2, 3, 1), overlap=5,
                     exchange_every=5, dt=W.dt_for(n, 2), tol=0.0, max_steps=77,
                     precision="fp64")
    ref = oracle.solve(prob)
    x1, _, _ = pma.solve(prob, want_psi=False, launch_mode=pma.PMA_LAUNCH_PER_SUBDOMAIN)
    assert _err(x1, ref, prob) <= 1e-11
    alone, _, _ = pma.solve(prob.replace(precision="fp32"), want_psi=False)
    others = W.config4(count=6, max_steps=50, size_range=(17, 97))
    res = pma.solve_many(others[:3] + [prob.replace(precision="fp32")] + others[3:])
    np.testing.assert_array_equal(res[3][0], alone)


def test_negative_exchange_every_is_rejected():
    prob = W.small_case(2, 21, parts=(2, 1, 1), overlap=4, steps=5).replace(exchange_every=-1)
    with pytest.raises(pma.PmaError) as e:
        pma.solve(prob)
    assert e.value.status == pma.PMA_ERR_INVALID
