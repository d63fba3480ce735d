"""Brute force on tiny grids: the oracle against a second, independent
implementation of the method, written out here at 50 significant digits.

The brute force restates the discretisation from its definitions and shares
nothing with the oracle's C code:
  * it works on Psi itself (not the deviation potential), in mpmath at 50
    digits, so no cancellation can hide an error;
  * every subdomain is a map from global node index to value;
  * the Neumann condition grad Psi . n = xi . n of Eq. (nbd) is imposed by
    its centred discretisation at a face, Psi_{-1} = Psi_1 - 2 h xi_0 (and
    Psi_N = Psi_{N-2} + 2 h xi_{N-1}), applied once per axis that leaves the
    box;
  * x = grad_h Psi and D_h^2 Psi are the centred differences of Eqs.
    (pmae1d)/(pmae2d); det D_h^2 Psi is mpmath's determinant;
  * the right-hand side is Eq. (pmae) with the density normalised by
    theta = sum over global nodes of the trapezoid-weighted rho det taken on
    the node's owner (the discrete int rho of Eq. edp), or the d-th-root form
    with theta of this or of the previous step;
  * transmission nodes follow Eq. (transmission_condition3) (owner's old
    value) or Algorithm 1 (owner's new value when the owner comes first in
    raster order), at every K-th step with the data frozen in between (the
    Delta tau intervals of Sect. 3);
  * the residual is max |Psi_tau| or the L2 increment of Eq.
    (dd_stop_criterion) per subdomain, combined by the max (every subdomain
    below tol) or by the min of Algorithm 1 step 6.
Each case runs a few steps on grids of at most 9 x 7 and 5^3 nodes, with
one or several subdomains, and compares the combined mesh, the combined Psi,
the residual of every step, the step count and the status.  CPU only.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2006_14602_gb300 import workloads as W

mp = pytest.importorskip("mpmath").mp
mp.dps = 50


# ------------------------------------------------------------------ density

def _rho(mon, x):
    """Monitor density at the point x (a tuple of mpf), from the term
    shapes of the problem description."""
    def term(t):
        if t.type == "bump":
            return t.amp * mp.exp(-t.width * sum((x[a] - t.c[a]) ** 2 for a in range(len(x))))
        if t.type == "ring":
            q = sum((x[a] - t.c[a]) ** 2 for a in range(len(x)))
            return t.amp * mp.exp(-t.width * (q - t.r2) ** 2)
        if t.type == "sine":
            s = x[t.axis] - t.c[t.axis] - t.a * mp.sin(2 * mp.pi * t.k * x[t.along])
            return t.amp * mp.exp(-t.width * s * s)
        if t.type == "bump1":
            return t.amp * mp.exp(-t.width * (x[t.axis] - t.c[t.axis]) ** 2)
        raise ValueError(t.type)
    if mon.kind == "sum":
        return mp.mpf(mon.base) + sum((term(t) for t in mon.terms), mp.mpf(0))
    if mon.kind == "product":
        r = mp.mpf(1)
        for t in mon.terms:
            r *= mon.base + term(t)
        return r
    raise ValueError(mon.kind)


# ------------------------------------------------------------ decomposition

def _parts_1d(N, p, o):
    """Cores [b_k, b_{k+1} - 1] with b_k = k N / p rounded half up; part k
    reaches floor(o/2) nodes below its core and ceil(o/2) above it (clipped
    at the ends of the axis)."""
    b = [int(mp.floor(mp.mpf(k * N) / p + mp.mpf(1) / 2)) for k in range(p + 1)]
    out = []
    for k in range(p):
        lo = 0 if k == 0 else b[k] - o // 2
        hi = N - 1 if k == p - 1 else b[k + 1] - 1 + (o - o // 2)
        out.append((lo, hi, b[k], b[k + 1] - 1))
    return out


class Brute:
    def __init__(self, prob, psi0=None):
        self.p = prob
        d = prob.dim
        self.d = d
        self.N = [int(prob.n[a]) for a in range(d)]
        self.lo = [mp.mpf(prob.lo[a]) for a in range(d)]
        self.h = [(mp.mpf(prob.hi[a]) - mp.mpf(prob.lo[a])) / (self.N[a] - 1) for a in range(d)]
        self.vol = mp.mpf(1)
        for a in range(d):
            self.vol *= mp.mpf(prob.hi[a]) - mp.mpf(prob.lo[a])
        ax = [_parts_1d(self.N[a], int(prob.parts[a]), int(prob.overlap)) for a in range(d)]
        self.pcount = [len(ax[a]) for a in range(d)]
        # subdomains in raster order (first axis fastest)
        self.subs = []
        for kk in itertools.product(*[range(len(ax[a])) for a in reversed(range(d))]):
            k = tuple(reversed(kk))
            box = [ax[a][k[a]] for a in range(d)]
            nodes = list(itertools.product(*[range(box[a][0], box[a][1] + 1) for a in range(d)]))
            inner = set()
            for g in nodes:
                for a in range(d):
                    if (g[a] == box[a][0] and k[a] > 0) or \
                       (g[a] == box[a][1] and k[a] < self.pcount[a] - 1):
                        inner.add(g)
            self.subs.append({"k": k, "box": box, "nodes": nodes, "dir": inner})
        # Psi^0 = |xi|^2 / 2 (Eq. incond) or the warm start
        self.psi = []
        for s in self.subs:
            m = {}
            for g in s["nodes"]:
                if psi0 is None:
                    m[g] = sum(self.xi(a, g[a]) ** 2 for a in range(d)) / 2
                else:
                    m[g] = mp.mpf(float(psi0[tuple(reversed(g))]))
            self.psi.append(m)
        self.theta_prev = None

    def xi(self, a, i):
        return self.lo[a] + i * self.h[a]

    def owner(self, g):
        for si, s in enumerate(self.subs):
            if all(s["box"][a][2] <= g[a] <= s["box"][a][3] for a in range(self.d)):
                return si
        raise AssertionError("no owner")

    def val(self, si, psi, g):
        """Psi of subdomain si at g; off the physical faces of Omega_c the
        discrete Neumann condition gives the ghost value."""
        for a in range(self.d):
            if g[a] < 0:
                inside = list(g)
                inside[a] = -g[a]
                return self.val(si, psi, tuple(inside)) - 2 * self.h[a] * self.xi(a, 0)
            if g[a] > self.N[a] - 1:
                inside = list(g)
                inside[a] = 2 * (self.N[a] - 1) - g[a]
                return self.val(si, psi, tuple(inside)) + 2 * self.h[a] * self.xi(a, self.N[a] - 1)
        return psi[si][g]

    def op(self, si, psi, g):
        """Mesh point and FD Hessian of Psi at global node g of subdomain si."""
        d = self.d
        def at(off):
            return self.val(si, psi, tuple(g[a] + off[a] for a in range(d)))
        e = [tuple(1 if b == a else 0 for b in range(d)) for a in range(d)]
        neg = lambda t: tuple(-q for q in t)
        add = lambda s, t: tuple(p + q for p, q in zip(s, t))
        zero = (0,) * d
        x = [(at(e[a]) - at(neg(e[a]))) / (2 * self.h[a]) for a in range(d)]
        H = mp.matrix(d, d)
        for a in range(d):
            H[a, a] = (at(e[a]) - 2 * at(zero) + at(neg(e[a]))) / self.h[a] ** 2
            for b in range(a + 1, d):
                H[a, b] = (at(add(e[a], e[b])) - at(add(e[a], neg(e[b]))) -
                           at(add(neg(e[a]), e[b])) + at(add(neg(e[a]), neg(e[b])))) / \
                          (4 * self.h[a] * self.h[b])
                H[b, a] = H[a, b]
        return x, H

    def weight(self, g, box=None):
        """Trapezoid weight, on the global grid or on a subdomain's box."""
        w = mp.mpf(1)
        for a in range(self.d):
            lo, hi = (0, self.N[a] - 1) if box is None else (box[a][0], box[a][1])
            w *= self.h[a] / 2 if g[a] in (lo, hi) else self.h[a]
        return w

    def step(self, n):
        """One forward-Euler step from Psi^n; returns (residual, tangled)."""
        p, d = self.p, self.d
        rd = {}
        for si, s in enumerate(self.subs):
            for g in s["nodes"]:
                if g in s["dir"]:
                    continue
                x, H = self.op(si, self.psi, g)
                D = mp.det(H)
                if not D > 0:
                    return None, True
                rd[(si, g)] = (_rho(p.monitor, x), D)
        theta = mp.mpf(0)
        for g in itertools.product(*[range(self.N[a]) for a in range(d)]):
            r, D = rd[(self.owner(g), g)]
            theta += self.weight(g) * r * D
        if self.theta_prev is None:
            self.theta_prev = theta
        new = [dict(m) for m in self.psi]
        res = []
        for si, s in enumerate(self.subs):
            fmax, l2 = mp.mpf(0), mp.mpf(0)
            for g in s["nodes"]:
                if g in s["dir"]:
                    continue
                r, D = rd[(si, g)]
                if p.rhs == "log":
                    F = mp.log(r * D)
                    if p.normalize == "global_theta":
                        F -= mp.log(theta / self.vol)
                else:
                    th = self.theta_prev if p.lag_theta else theta
                    z = r * D * (self.vol / th if p.normalize == "global_theta" else 1)
                    F = mp.power(z, mp.mpf(1) / d) - 1
                new[si][g] = self.psi[si][g] + p.dt * F
                fmax = max(fmax, abs(F))
                l2 += self.weight(g, s["box"]) * (new[si][g] - self.psi[si][g]) ** 2
            res.append(fmax if p.stop_norm == "max_ut" else mp.sqrt(l2))
        K = max(1, int(p.exchange_every))
        if n % K == 0:
            for si, s in enumerate(self.subs):
                for g in s["dir"]:
                    o = self.owner(g)
                    src = new if (p.alternating and o < si) else self.psi
                    new[si][g] = src[o][g]
        self.theta_prev = theta
        self.psi = new
        return (max(res) if p.stop_rule == "all" else min(res)), False

    def run(self):
        p = self.p
        hist, steps, status = [], 0, "not_converged"
        for n in range(int(p.max_steps)):
            r, tangled = self.step(n)
            if tangled:
                status = "tangled"
                break
            hist.append(r)
            steps = n + 1
            if steps % max(1, int(p.check_every)) == 0 and r <= p.tol:
                status = "ok"
                break
        return hist, steps, status

    def mesh(self):
        """Owner-takes combination on the global grid, arrays (z, y, x)."""
        d = self.d
        shape = tuple(reversed(self.N))
        X = np.zeros((d,) + shape)
        P = np.zeros(shape)
        for g in itertools.product(*[range(self.N[a]) for a in range(d)]):
            o = self.owner(g)
            x, _ = self.op(o, self.psi, g)
            for a in range(d):
                X[(a,) + tuple(reversed(g))] = float(x[a])
            P[tuple(reversed(g))] = float(self.psi[o][g])
        return X, P


# ------------------------------------------------------------------ cases

def _ring(dim):
    return W.ring_monitor(dim, amp=10.0, width=50.0, r2=0.06, centre=(0.45, 0.55, 0.5))


def _cases():
    two = dict(dim=2, n=(9, 7, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 0.8, 1.0))
    blocks = dict(dim=2, n=(7, 7, 1), lo=(-0.2, 0.1, 0.0), hi=(0.9, 1.3, 1.0))
    cube = dict(dim=3, n=(5, 5, 5))
    sine = W.sine_monitor()
    bumps = W.Monitor("sum", 1.0, [W.Term("bump", 8.0, 30.0, 0.0, (0.3, 0.6, 0.5)),
                                    W.Term("ring", 5.0, 40.0, 0.05, (0.6, 0.4, 0.5))])
    prod = W.product_monitor([(4.0, 20.0, 0.3), (2.0, 15.0, 0.7)])
    C = {
        "1d_single": dict(dim=1, n=(9, 1, 1), monitor=W.Monitor(
            "sum", 1.0, [W.Term("bump", 6.0, 40.0, 0.0, (0.4, 0.5, 0.5))])),
        "1d_slabs_l2": dict(dim=1, n=(9, 1, 1), parts=(2, 1, 1), overlap=3,
                            stop_norm="l2_increment", monitor=W.Monitor(
                                "sum", 1.0, [W.Term("bump", 6.0, 40.0, 0.0, (0.6, 0.5, 0.5))])),
        "2d_single_ring": dict(two, monitor=_ring(2)),
        "2d_slabs_parallel": dict(two, parts=(2, 1, 1), overlap=3, monitor=_ring(2)),
        "2d_slabs_alternating": dict(two, parts=(2, 1, 1), overlap=3, alternating=1,
                                     monitor=_ring(2)),
        "2d_blocks_parallel_any": dict(blocks, parts=(2, 2, 1), overlap=2, stop_rule="any",
                                       monitor=bumps),
        "2d_blocks_alternating_l2": dict(blocks, parts=(2, 2, 1), overlap=3, alternating=1,
                                         stop_norm="l2_increment", monitor=bumps),
        "2d_blocks_root": dict(blocks, parts=(2, 2, 1), overlap=2, rhs="root", monitor=sine),
        "2d_blocks_root_lagged": dict(blocks, parts=(2, 2, 1), overlap=2, rhs="root",
                                      lag_theta=1, monitor=bumps),
        "2d_blocks_unnormalised": dict(blocks, parts=(2, 2, 1), overlap=2, normalize="none",
                                       monitor=prod),
        "2d_blocks_exchange2": dict(blocks, parts=(2, 2, 1), overlap=3, exchange_every=2,
                                    monitor=bumps),
        "2d_slabs_alternating_exchange3": dict(two, parts=(2, 1, 1), overlap=3, alternating=1,
                                               exchange_every=3, monitor=_ring(2)),
        "3d_single_shell": dict(cube, monitor=_ring(3)),
        "3d_blocks_parallel": dict(cube, parts=(2, 2, 2), overlap=2, monitor=_ring(3)),
        "3d_blocks_alternating_root": dict(cube, parts=(2, 1, 2), overlap=2, alternating=1,
                                           rhs="root", monitor=_ring(3)),
        "3d_slabs_exchange2_l2_any": dict(cube, parts=(1, 2, 1), overlap=2, exchange_every=2,
                                          stop_norm="l2_increment", stop_rule="any",
                                          monitor=_ring(3)),
    }
    return C


CASES = _cases()


def _problem(name, steps=3):
    kw = dict(CASES[name])
    dim = kw["dim"]
    n, lo, hi = kw["n"], kw.get("lo", (0.0,) * 3), kw.get("hi", (1.0,) * 3)
    h2 = min(((hi[a] - lo[a]) / (n[a] - 1)) ** 2 for a in range(dim))
    kw.setdefault("dt", 0.1 * h2)
    kw.setdefault("tol", 0.0)
    kw.setdefault("max_steps", steps)
    return W.Problem(**kw)


def _warm_start(prob, seed):
    """|xi|^2/2 plus a small random perturbation (det stays positive)."""
    rng = np.random.default_rng(seed)
    xs = [np.linspace(prob.lo[a], prob.hi[a], prob.n[a]) for a in range(prob.dim)]
    G = np.meshgrid(*xs, indexing="ij")
    h2 = min(((prob.hi[a] - prob.lo[a]) / (prob.n[a] - 1)) ** 2 for a in range(prob.dim))
    psi = sum(0.5 * g * g for g in G) + 0.04 * h2 * rng.uniform(-1, 1, size=G[0].shape)
    return np.ascontiguousarray(psi.T)


def check_case(name, warm=False, steps=3):
    prob = _problem(name, steps)
    psi0 = _warm_start(prob, 11) if warm else None
    b = Brute(prob, psi0)
    hist, nsteps, status = b.run()
    X, P = b.mesh()
    r = oracle.solve(prob, psi0=psi0)
    assert r.steps == nsteps and r.status == status, (name, r.steps, nsteps, r.status, status)
    size = max(prob.hi[a] - prob.lo[a] for a in range(prob.dim))
    assert np.abs(r.x - X).max() <= 1e-13 * size, (name, np.abs(r.x - X).max())
    assert np.abs(r.psi - P).max() <= 1e-13, (name, np.abs(r.psi - P).max())
    want = np.array([float(v) for v in hist])
    assert np.allclose(r.res, want, rtol=1e-10, atol=1e-300), (name, r.res, want)


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_equals_brute_force(name):
    check_case(name)


@pytest.mark.parametrize("name", ["2d_blocks_alternating_l2", "3d_blocks_parallel",
                                  "2d_blocks_root_lagged", "2d_blocks_exchange2"])
def test_oracle_equals_brute_force_from_warm_start(name):
    check_case(name, warm=True)


def test_brute_force_stop_rule_and_check_every():
    """The stop decision itself: a tolerance between the residuals of steps
    2 and 4 stops at the first checked step below it."""
    prob = _problem("2d_blocks_parallel_any", steps=6)
    hist, _, _ = Brute(prob).run()
    tol = float((hist[2] + hist[3]) / 2)
    for ce in (1, 2, 3):
        p = prob.replace(tol=tol, check_every=ce)
        hb, nb, sb = Brute(p).run()
        r = oracle.solve(p)
        assert (r.steps, r.status) == (nb, sb)
        assert sb == "ok" or nb == 6


def check_all():
    """Every case once (the planted-mistake tests call this)."""
    for name in sorted(CASES):
        check_case(name)
