"""Seeded random problems against the FP64 oracle: every option of the
problem statement drawn at random (2D / 3D, grid sizes and domains,
decompositions and overlaps, parallel or alternating transmission,
exchange_every, log or root form, both stop norms and rules, check_every,
normalisation on or off, monitor kinds (bump/ring sums, separable
products, tables, an arc-length density), warm starts, FP64 or FP32), all
of them in one
batched context next to each other, each compared node by node with the
oracle after the same steps (FP64 1e-11, FP32 1e-5 of the domain size) with
the same step count and status."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_14602_gb300 import pma
from paper_2006_14602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _parts(rng, n, o):
    # largest admissible count: every core holds at least ceil(o/2) + 2 nodes
    pmax = max(1, min(4, n // (o // 2 + o - o // 2 + 3)))
    return int(rng.integers(1, pmax + 1))


def _problem(rng):
    dim = 2 if rng.uniform() < 0.7 else 3
    side = (9, 48) if dim == 2 else (7, 20)
    n = [int(rng.integers(side[0], side[1])) for _ in range(dim)]
    lo = [float(rng.uniform(-0.5, 0.5)) for _ in range(dim)]
    hi = [lo[a] + float(rng.uniform(0.6, 1.6)) for a in range(dim)]
    o = int(rng.integers(2, 7))
    parts = [_parts(rng, n[a], o) for a in range(dim)]
    if all(p == 1 for p in parts):
        o = 0
    centre = tuple(lo[a] + 0.5 * (hi[a] - lo[a]) for a in range(dim)) + (0.5,) * (3 - dim)
    kind = rng.integers(0, 5)
    if kind == 3:
        # a tabulated density on its own box (clamped outside), values from a
        # smooth positive function
        tn = [int(rng.integers(4, 12)) for _ in range(dim)]
        tlo = [lo[a] - 0.1 for a in range(dim)]
        thi = [hi[a] + 0.05 for a in range(dim)]
        axes = [np.linspace(tlo[a], thi[a], tn[a]) for a in range(dim)]
        G = np.meshgrid(*axes, indexing="ij")
        phase = rng.uniform(0, 2 * math.pi, size=dim)
        val = 1.5 + sum(0.6 * np.cos(2.5 * g + ph) for g, ph in zip(G, phase)) / dim
        mon = W.Monitor(kind="table", table=np.ascontiguousarray(val.T),
                        tlo=tuple(tlo) + (0.0,) * (3 - dim), thi=tuple(thi) + (1.0,) * (3 - dim))
    elif kind == 4 and dim == 2:
        mon = W.Monitor("arclen_burgers", 1.0, [], p0=float(rng.uniform(0.08, 0.2)))
    elif kind in (0, 4):
        mon = W.random_bumps(rng, dim)
        # centres inside this problem's box
        for t in mon.terms:
            t.c = tuple(lo[a] + (t.c[a] - 0.2) / 0.6 * (hi[a] - lo[a]) if a < dim else 0.5
                        for a in range(3))
    elif kind == 1:
        mon = W.ring_monitor(dim, amp=float(rng.uniform(2, 12)), width=float(rng.uniform(10, 60)),
                             r2=float(rng.uniform(0.01, 0.06)), centre=centre)
    else:
        f = [(float(rng.uniform(1, 5)), float(rng.uniform(5, 30)),
              lo[a] + float(rng.uniform(0.3, 0.7)) * (hi[a] - lo[a])) for a in range(dim)]
        mon = W.product_monitor(f)
    rhs = "root" if rng.uniform() < 0.25 else "log"
    prec = str(rng.choice(["fp64", "fp32"]))
    # a tolerance only where both sides see the same residual to rounding
    tol = float(rng.choice([0.0, 1e-3])) if prec == "fp64" else 0.0
    nn = tuple(n) + (1,) * (3 - dim)
    cfl = (0.06 if dim == 2 else 0.03) * float(rng.uniform(0.5, 1.0))
    h2 = min(((hi[a] - lo[a]) / (n[a] - 1)) ** 2 for a in range(dim))
    return W.Problem(
        dim=dim, n=nn, lo=tuple(lo) + (0.0,) * (3 - dim), hi=tuple(hi) + (1.0,) * (3 - dim),
        monitor=mon, parts=tuple(parts) + (1,) * (3 - dim), overlap=o,
        alternating=int(rng.uniform() < 0.3), exchange_every=int(rng.choice([1, 1, 2, 3])),
        dt=cfl * h2, tol=tol,
        max_steps=int(rng.integers(5, 90)),
        stop_norm=str(rng.choice(["max_ut", "l2_increment"])),
        stop_rule=str(rng.choice(["all", "any"])), check_every=int(rng.choice([1, 1, 3])),
        rhs=rhs, lag_theta=1 if rhs == "root" else 0,
        normalize="none" if rng.uniform() < 0.2 else "global_theta",
        precision=prec)


def _warm_start(rng, p):
    """|xi|^2/2 plus a small smooth perturbation (a previous steady state
    stand-in, Sect. 2), or None."""
    if rng.uniform() < 0.7:
        return None
    axes = [np.linspace(p.lo[a], p.hi[a], p.n[a]) for a in range(p.dim)]
    G = np.meshgrid(*axes, indexing="ij")
    h2 = min(((p.hi[a] - p.lo[a]) / (p.n[a] - 1)) ** 2 for a in range(p.dim))
    bump = sum(np.cos(math.pi * (g - p.lo[a]) / (p.hi[a] - p.lo[a])) for a, g in enumerate(G))
    return np.ascontiguousarray((sum(0.5 * g * g for g in G) + 0.02 * bump *
                                 (max(p.hi[a] - p.lo[a] for a in range(p.dim)) ** 2) / p.dim).T)


def test_random_problems_in_one_batch():
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()
    rng = np.random.default_rng(20061460)
    probs = [_problem(rng) for _ in range(64)]
    psi0s = [_warm_start(rng, p) for p in probs]
    refs = oracle.solve_parallel([p.replace(precision="fp64") for p in probs], psi0s=psi0s)
    with pma.Context(window_steps=16) as ctx:
        ids = [ctx.submit(p, q) for p, q in zip(probs, psi0s)]
        ctx.run()
        res = [ctx.mesh(p, i) for p, i in zip(probs, ids)]
    kinds = set()
    for i, (p, ref, (x, _, info)) in enumerate(zip(probs, refs, res)):
        kinds.add((p.dim, p.precision, p.alternating, p.exchange_every > 1, p.rhs,
                   p.monitor.kind))
        if p.precision == "fp64" or ref.status != "tangled":
            assert info.steps == ref.steps, (i, info.steps, ref.steps)
        if p.precision == "fp64":
            assert pma.STATUS_NAMES[info.status] == ref.status, i
        size = max(p.hi[a] - p.lo[a] for a in range(p.dim))
        tol = 1e-11 if p.precision == "fp64" else 1e-5
        if ref.status != "tangled":
            assert np.abs(x - ref.x).max() <= tol * size, (i, np.abs(x - ref.x).max())
    assert len(kinds) >= 20


def test_random_problems_in_every_execution_mode():
    """The same random problems through the other execution paths: one
    launch per subdomain and step without graphs, two request groups on two
    streams, and graphs off must give the batched path's bits; the
    cluster-resident path (a different summation order of theta) and the
    allocation-free entry point must meet the oracle bounds."""
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()
    rng = np.random.default_rng(1460620)
    probs = [_problem(rng) for _ in range(24)]
    refs = oracle.solve_parallel([p.replace(precision="fp64") for p in probs])

    def run(**opts):
        with pma.Context(window_steps=8, **opts) as ctx:
            ids = [ctx.submit(p) for p in probs]
            ctx.run()
            return [ctx.mesh(p, i) for p, i in zip(probs, ids)]

    base = run()
    for opts in ({"launch_mode": pma.PMA_LAUNCH_PER_SUBDOMAIN, "use_graphs": 0},
                 {"groups": 2}, {"use_graphs": 0}):
        for (a, _, ia), (b, _, ib) in zip(base, run(**opts)):
            assert ia.steps == ib.steps and ia.status == ib.status, opts
            np.testing.assert_array_equal(a, b, err_msg=str(opts))
    for i, (p, ref, (x, _, info)) in enumerate(zip(probs, refs, run(resident=4))):
        size = max(p.hi[a] - p.lo[a] for a in range(p.dim))
        tol = 1e-11 if p.precision == "fp64" else 1e-5
        if ref.status != "tangled":
            assert info.steps == ref.steps
            assert np.abs(x - ref.x).max() <= tol * size, (i, "resident")
    for i, (p, ref) in enumerate(zip(probs, refs)):
        if ref.status == "tangled":
            continue
        g, m, d, q = pma.to_structs(p)
        out = torch.empty(p.dim * p.nodes, dtype=torch.float64, device="cuda")
        st, info = pma.pma_solve_static(g, m, d, q, 0, out.data_ptr(), 0)
        assert st in (pma.PMA_OK, pma.PMA_NOT_CONVERGED), (i, pma.pma_last_error())
        assert info.steps == ref.steps
        x = out.cpu().numpy().reshape(ref.x.shape)
        size = max(p.hi[a] - p.lo[a] for a in range(p.dim))
        tol = 1e-11 if p.precision == "fp64" else 1e-5
        assert np.abs(x - ref.x).max() <= tol * size, (i, "static")
