"""The paper's Sect. 4 studies, run on the device path (FP64).

  * space convergence of the DD steady state (Sect. 4.4, Figure
    dd_convergence): 4 subdomains at 65^2, 129^2 and 257^2; without a
    finer single-domain reference (forward Euler needs ~N^2 steps to reach
    the steady state, several million at 1025^2) the order comes from the
    nested grids: the differences 65->129 and 129->257 at the common nodes
    shrink by 2^p, p ~ 2 (paper: 1.85, 2.01, 1.99);
  * convergence history (Figure dd_convergencetx): the DD solution tends to
    the single-domain steady state of the same grid as the step count grows;
  * overlap study (Figure dd_convergencetxx): after a fixed number of
    steps the DD-vs-SD error falls as the overlap grows (5, 9, 11, 15);
  * Table quality_measure_table: E_2 of the whole-domain, 4-slab and 2x2
    block meshes at 21^2 and 41^2 within 1 % of the printed values, and
    equal to the oracle's E_2 of the same problem.
The ring density stands in for the spiral of Eq. (test_fn2), whose density
(up to ~1600) tangles explicit Euler on these grids; the quality table uses
the Burgers-front arc-length density of Eq. (test_fn1).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2006_14602_gb300 import pma
from paper_2006_14602_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()


def _steady(n, parts=(2, 2, 1), overlap=4, tol=1e-9):
    return W.Problem(dim=2, n=(n, n, 1), monitor=W.ring_monitor(), parts=parts,
                     overlap=overlap if parts != (1, 1, 1) else 0,
                     dt=W.dt_for((n, n, 1), 2), tol=tol, max_steps=10 ** 7, precision="fp64")


def test_space_convergence_second_order_on_the_device():
    gold = json.load(open(os.path.join(GOLD, "convergence_slopes.json")))
    xs = {}
    for n in (65, 129, 257):
        x, _, info = pma.solve(_steady(n), want_psi=False, window_steps=256)
        assert pma.STATUS_NAMES[info.status] == "ok", (n, info.steps, info.residual)
        s = (n - 1) // 64
        xs[n] = x[:, ::s, ::s]
    d1, d2 = xs[65] - xs[129], xs[129] - xs[257]
    orders = {}
    for name, norm in (("L1", lambda d: np.abs(d).sum()), ("L2", lambda d: math.sqrt((d * d).sum())),
                       ("Linf", lambda d: np.abs(d).max())):
        orders[name] = math.log2(norm(d1) / norm(d2))
    for name, p in orders.items():
        assert 1.7 <= p <= 2.3, orders
        assert abs(p - gold["space_slopes"][name]) < 0.35, orders


def test_steady_state_65_equals_the_oracle():
    prob = _steady(65)
    ref = oracle.solve(prob)
    x, _, info = pma.solve(prob, want_psi=False, window_steps=256)
    assert info.steps == ref.steps and pma.STATUS_NAMES[info.status] == ref.status == "ok"
    assert np.abs(x - ref.x).max() <= 1e-11


def test_convergence_history_and_overlap_study():
    n = 129
    sd, _, _ = pma.solve(_steady(n, parts=(1, 1, 1)), want_psi=False, window_steps=256)
    base = _steady(n).replace(tol=0.0)
    # history: the DD mesh approaches the single-domain steady state
    hist = []
    for steps in (1000, 4000, 16000, 64000):
        x, _, _ = pma.solve(base.replace(max_steps=steps), want_psi=False, window_steps=256)
        hist.append(np.abs(x - sd).max())
    assert all(a > b for a, b in zip(hist, hist[1:])), hist
    assert hist[-1] < 1e-6
    # overlap: at a fixed step count the error falls as the overlap grows
    sd1k, _, _ = pma.solve(_steady(n, parts=(1, 1, 1)).replace(tol=0.0, max_steps=1000),
                           want_psi=False)
    gold = json.load(open(os.path.join(GOLD, "convergence_slopes.json")))
    errs = []
    for o in [3] + gold["overlap_points"]:
        x, _, _ = pma.solve(base.replace(max_steps=1000, overlap=o), want_psi=False)
        errs.append(np.abs(x - sd1k).max())
    assert all(a > b for a, b in zip(errs, errs[1:])), errs


def _e2(x, n, mon):
    X, Y = x
    h = 1.0 / (n - 1)
    J = (np.gradient(X, h, axis=1) * np.gradient(Y, h, axis=0) -
         np.gradient(X, h, axis=0) * np.gradient(Y, h, axis=1))
    rho = oracle.monitor_eval(mon, 2, np.stack([X.ravel(), Y.ravel()], 1)).reshape(X.shape)
    w = np.full((n, n), h * h)
    w[[0, -1], :] *= 0.5
    w[:, [0, -1]] *= 0.5
    E = rho * J / (w * rho * J).sum()
    return math.sqrt((w * E * E).sum() / w.sum())


def test_quality_table_from_device_meshes():
    gold = json.load(open(os.path.join(GOLD, "quality_table.json")))["rows"]
    mon = W.Monitor("arclen_burgers", 1.0, [], p0=0.01)
    rows = {"whole domain": ((1, 1, 1), 0), "4 slabs DD": ((4, 1, 1), 3),
            "2x2 block DD": ((2, 2, 1), 3)}
    probs, keys = [], []
    for n in (21, 41):
        for row, (parts, o) in rows.items():
            probs.append(W.Problem(dim=2, n=(n, n, 1), monitor=mon, parts=parts, overlap=o,
                                   dt=W.dt_for((n, n, 1), 2, cfl=0.02), tol=1e-6,
                                   max_steps=10 ** 6, precision="fp64"))
            keys.append((n, row))
    refs = oracle.solve_parallel(probs)
    for (n, row), prob, ref in zip(keys, probs, refs):
        x, _, info = pma.solve(prob, want_psi=False, window_steps=256)
        assert info.steps == ref.steps and pma.STATUS_NAMES[info.status] == "ok"
        e_dev, e_ref = _e2(x, n, mon), _e2(ref.x, n, mon)
        assert abs(e_dev - e_ref) < 1e-9, (n, row, e_dev, e_ref)
        assert abs(e_dev - gold[row][str(n)]["E2"]) < 0.01 * gold[row][str(n)]["E2"], (n, row, e_dev)
