"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares it with an
independent fact -- a closed form, an invariant of the discretisation, a
reduction to a 1D problem solved by quadrature, a symmetry, or a behaviour
the paper reports (Sects. 2-4).  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
from paper_2006_14602_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _xi(prob):
    """Node coordinates per axis."""
    return [np.linspace(prob.lo[a], prob.hi[a], prob.n[a]) for a in range(prob.dim)]


def _identity(prob):
    xs = _xi(prob)
    grids = np.meshgrid(*xs, indexing="ij")
    # oracle arrays are (z, y, x): reverse axis order
    return np.stack([g.T for g in grids])


# ---------------------------------------------------------------- monitors

def test_monitor_closed_forms():
    ring = W.ring_monitor()  # 1 + 10 exp(-50 (|x-c|^2 - 0.0625)^2)
    pts = np.array([[0.75, 0.5], [0.5, 0.25], [0.5, 0.5], [0.0, 0.0]])
    got = oracle.monitor_eval(ring, 2, pts)
    want = [11.0, 11.0, 1 + 10 * math.exp(-50 * 0.0625 ** 2),
            1 + 10 * math.exp(-50 * (0.5 - 0.0625) ** 2)]
    np.testing.assert_allclose(got, want, rtol=1e-14)
    sine = W.sine_monitor()  # 1 + 5 exp(-100 (x2 - 0.5 - 0.25 sin(2 pi x1))^2)
    got = oracle.monitor_eval(sine, 2, np.array([[0.0, 0.5], [0.25, 0.75], [0.75, 0.25],
                                                 [0.25, 0.5]]))
    np.testing.assert_allclose(got, [6.0, 6.0, 6.0, 1 + 5 * math.exp(-100 * 0.0625)],
                               rtol=1e-14)
    shell = W.shell_monitor()
    got = oracle.monitor_eval(shell, 3, np.array([[0.8, 0.5, 0.5], [0.5, 0.5, 0.5]]))
    np.testing.assert_allclose(got, [21.0, 1 + 20 * math.exp(-80 * 0.09 ** 2)], rtol=1e-14)
    prod = W.product_monitor([(3.0, 40.0, 0.3), (2.0, 10.0, 0.6)])
    x = np.array([[0.3, 0.6], [0.1, 0.9]])
    want = [(1 + 3) * (1 + 2),
            (1 + 3 * math.exp(-40 * 0.04)) * (1 + 2 * math.exp(-10 * 0.09))]
    np.testing.assert_allclose(oracle.monitor_eval(prod, 2, x), want, rtol=1e-14)
    unif = W.uniform_monitor(2.5)
    assert np.all(oracle.monitor_eval(unif, 3, np.random.rand(5, 3)) == 2.5)


def _u_burgers(x, y, eps):
    return 1.0 / (1.0 + np.exp((x + y - 1.0) / (2 * eps)))


def _u_spiral(x, y):
    r2 = (x - 0.7) ** 2 + (y - 0.5) ** 2
    th = np.arctan2(y - 0.5, x - 0.7)
    return 1.0 + 9.0 / (1.0 + 100.0 * r2 * np.cos(th - 20.0 * r2) ** 2)


def _u_tanh(x, y, z):
    return np.tanh(100.0 * (x * x + y * y + z * z - 0.125))


def _u_nine(x, y, z):
    c = [(0, 0, 0), (.5, .5, .5), (.5, -.5, .5), (-.5, .5, .5), (-.5, -.5, .5),
         (.5, .5, -.5), (.5, -.5, -.5), (-.5, .5, -.5), (-.5, -.5, -.5)]
    return sum(np.tanh(50.0 * ((x - a) ** 2 + (y - b) ** 2 + (z - d) ** 2 - 0.1875))
               for a, b, d in c)


@pytest.mark.parametrize("kind", ["arclen_burgers", "arclen_spiral", "arclen_tanh_sphere",
                                  "arclen_nine_spheres"])
def test_arclength_monitors_match_numerical_gradient(kind):
    """Eq. (monitfn): rho = sqrt(1 + |grad u|^2), with grad u of the test
    functions (Eqs. test_fn1/test_fn2/test_fn3d1/test_fn3d2) taken here by
    Richardson-extrapolated central differences of u itself."""
    rng = np.random.default_rng(3)
    eps = 0.05
    mon = W.Monitor(kind, 1.0, [], p0=eps)
    if kind in ("arclen_burgers", "arclen_spiral"):
        dim = 2
        pts = rng.uniform(0.0, 1.0, size=(40, 2))
        if kind == "arclen_spiral":
            pts = pts[np.hypot(pts[:, 0] - 0.7, pts[:, 1] - 0.5) > 0.05]
            f = lambda p: _u_spiral(*p)
        else:
            f = lambda p: _u_burgers(*p, eps)
    else:
        dim = 3
        lim = 1.0 if kind == "arclen_tanh_sphere" else 2.0
        pts = rng.uniform(-lim, lim, size=(40, 3))
        if kind == "arclen_tanh_sphere":
            # keep the sech^2 shell resolvable by the difference quotient
            pts = pts * 0.45 + 0.0
            f = lambda p: _u_tanh(*p)
        else:
            f = lambda p: _u_nine(*p)
    want = []
    for p in pts:
        g = []
        for a in range(dim):
            def d(hh):
                e = np.zeros(dim)
                e[a] = hh
                return (f(p + e) - f(p - e)) / (2 * hh)
            hh = 1e-4
            g.append((4 * d(hh / 2) - d(hh)) / 3)
        want.append(math.sqrt(1 + sum(v * v for v in g)))
    got = oracle.monitor_eval(mon, dim, pts)
    np.testing.assert_allclose(got, want, rtol=2e-6)


# ---------------------------------------------------------------- operators

@pytest.mark.parametrize("dim", [1, 2, 3])
def test_operator_exact_on_quadratics(dim):
    """Centred differences (Eqs. pmae1d/pmae2d) are exact on quadratics: at
    nodes away from the faces, grad_h and D_h^2 of v = xi.A.xi/2 + b.xi give
    x = xi + A xi + b and det(I + A) exactly."""
    n = {1: 11, 2: 9, 3: 7}[dim]
    prob = W.Problem(dim=dim, n=(n, n if dim > 1 else 1, n if dim > 2 else 1),
                     lo=(-0.3, 0.2, 1.0), hi=(0.9, 1.7, 1.6), monitor=W.uniform_monitor())
    A = np.array([[0.31, -0.12, 0.07], [-0.12, 0.23, 0.05], [0.07, 0.05, -0.17]])[:dim, :dim]
    b = np.array([0.05, -0.02, 0.03])[:dim]
    xs = np.meshgrid(*_xi(prob), indexing="ij")
    X = np.stack(xs)  # (dim, nx, ny, nz) in ij order
    v = 0.5 * np.einsum("a...,ab,b...->...", X, A, X) + np.einsum("a,a...->...", b, X)
    x, det, rho, G = oracle.operator(prob, v.T.copy())
    want_x = X + np.einsum("ab,b...->a...", A, X) + b.reshape((dim,) + (1,) * dim)
    inner = (slice(1, -1),) * dim
    for a in range(dim):
        np.testing.assert_allclose(x[a][inner], want_x[a].T[inner], rtol=0, atol=1e-13)
    np.testing.assert_allclose(det[inner], np.linalg.det(np.eye(dim) + A), rtol=1e-12)
    np.testing.assert_allclose(rho, 1.0)
    np.testing.assert_allclose(G[inner], math.log(np.linalg.det(np.eye(dim) + A)), rtol=1e-11)


def test_neumann_mirror_keeps_boundary_nodes_on_boundary():
    """Eq. (nbd) / Eqs. (adapt_mesh_bc1-2): boundary nodes only slide along
    the boundary.  For a Neumann-compatible v the mirror ghost gives
    x_a = xi_a exactly on faces normal to a, and the second difference at a
    face converges to v'' at O(h^2)."""
    errs = []
    for n in (17, 33):
        prob = W.Problem(dim=2, n=(n, n, 1), monitor=W.uniform_monitor())
        xi, eta = np.meshgrid(*_xi(prob), indexing="xy")
        v = 0.02 * np.cos(math.pi * xi) * np.cos(2 * math.pi * eta) + 0.01 * np.cos(3 * math.pi * eta)
        x, det, _, _ = oracle.operator(prob, v)
        assert np.array_equal(x[0][:, 0], xi[:, 0]) and np.array_equal(x[0][:, -1], xi[:, -1])
        assert np.array_equal(x[1][0, :], eta[0, :]) and np.array_equal(x[1][-1, :], eta[-1, :])
        # det on the left face: (1 + v_xixi)(1 + v_etaeta) - 0 (mixed term vanishes)
        e = eta[:, 0]
        vxx = -0.02 * math.pi ** 2 * np.cos(2 * math.pi * e)
        vyy = (-0.02 * 4 * math.pi ** 2 * np.cos(2 * math.pi * e)
               - 0.01 * 9 * math.pi ** 2 * np.cos(3 * math.pi * e))
        errs.append(np.abs(det[:, 0] - (1 + vxx) * (1 + vyy)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_1d_trapezoid_sum_of_det_is_domain_length():
    """Discrete mass identity in 1D: with the mirror ghost and trapezoid
    weights, sum_i w_i D_h^2 Psi_i telescopes to |Omega_c| for any Psi."""
    rng = np.random.default_rng(7)
    n = 41
    prob = W.Problem(dim=1, n=(n, 1, 1), lo=(0.5, 0, 0), hi=(2.0, 1, 1),
                     monitor=W.uniform_monitor())
    v = 1e-3 * rng.standard_normal(n)
    _, det, _, _ = oracle.operator(prob, v)
    h = 1.5 / (n - 1)
    w = np.full(n, h)
    w[[0, -1]] *= 0.5
    assert abs((w * det).sum() - 1.5) < 1e-12


def test_extents_overlap_and_cores():
    """Sect. 3 decomposition: alpha^i < alpha^{i+1} < beta^i < beta^{i+1};
    neighbours share exactly `overlap` nodes; cores tile the axis; every
    transmission node lies in a neighbour's core, away from its edges."""
    for n, p, o in [(257, 4, 8), (129, 2, 6), (33, 4, 3), (65, 3, 5), (100, 7, 2)]:
        lo, hi, clo, chi = oracle.extents(n, p, o)
        assert lo[0] == 0 and hi[-1] == n - 1 and clo[0] == 0 and chi[-1] == n - 1
        assert np.all(clo[1:] == chi[:-1] + 1)
        for k in range(p - 1):
            assert lo[k] < lo[k + 1] < hi[k] < hi[k + 1]
            assert hi[k] - lo[k + 1] + 1 == o
            # transmission nodes: hi[k] is owned by k+1, lo[k+1] by k
            assert clo[k + 1] <= hi[k] <= chi[k + 1] and lo[k + 1] < hi[k] < hi[k + 1]
            assert clo[k] <= lo[k + 1] <= chi[k] and lo[k] < lo[k + 1] < hi[k]
    with pytest.raises(ValueError):
        oracle.extents(20, 4, 12)
    with pytest.raises(ValueError):
        oracle.extents(33, 2, 1)


# ---------------------------------------------------------------- P1

@pytest.mark.parametrize("dim,parts,overlap", [(1, (1, 1, 1), 0), (1, (3, 1, 1), 4),
                                               (2, (1, 1, 1), 0), (2, (2, 3, 1), 4),
                                               (3, (1, 1, 1), 0), (3, (2, 2, 2), 3)])
def test_uniform_density_keeps_identity(dim, parts, overlap):
    """Sect. 2: rho == const gives the identity map; Psi^0 = |xi|^2/2 of
    Eq. (incond) is then stationary."""
    n = {1: 31, 2: 19, 3: 11}[dim]
    prob = W.Problem(dim=dim, n=(n, n if dim > 1 else 1, n if dim > 2 else 1),
                     lo=(0.1, -0.4, 0.0), hi=(1.3, 0.6, 2.0), monitor=W.uniform_monitor(3.7),
                     parts=parts, overlap=overlap, dt=1e-4, tol=0.0, max_steps=500)
    r = oracle.solve(prob)
    assert r.status == "not_converged" and r.steps == 500
    np.testing.assert_allclose(r.x, _identity(prob), rtol=0, atol=1e-12)
    xs = np.meshgrid(*_xi(prob), indexing="ij")
    psi0 = sum(0.5 * g * g for g in xs).T
    np.testing.assert_allclose(r.psi, psi0, rtol=0, atol=1e-12)
    assert r.residual < 1e-12


# ---------------------------------------------------------------- P2

def _inverse_cdf(mon, lo, hi, xi):
    rho = lambda s: oracle.monitor_eval(mon, 1, np.array([s]))[0]
    total = integrate.quad(rho, lo, hi, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    out = []
    for t in xi:
        target = total * (t - lo) / (hi - lo)
        if t <= lo or t >= hi:
            out.append(t)
            continue
        f = lambda X: integrate.quad(rho, lo, X, epsabs=1e-14, epsrel=1e-13, limit=200)[0] - target
        out.append(optimize.brentq(f, lo, hi, xtol=1e-15, rtol=1e-15))
    return np.array(out)


def test_1d_steady_state_equidistributes():
    """Eq. (edp1)/(edp) in 1D: the steady state equidistributes rho, so
    x(xi) is the inverse of the normalised cumulative density; the discrete
    error is second order."""
    mon = W.Monitor("sum", 1.0, [W.Term("bump", 10.0, 50.0, 0.0, (0.4, 0.5, 0.5))])
    errs = []
    for n in (33, 65):
        prob = W.Problem(dim=1, n=(n, 1, 1), monitor=mon, dt=W.dt_for((n, 1, 1), 1, cfl=0.04),
                         tol=1e-11, max_steps=10 ** 6)
        r = oracle.solve(prob)
        assert r.status == "ok"
        xi = _xi(prob)[0]
        X = _inverse_cdf(mon, 0.0, 1.0, xi)
        errs.append(np.abs(r.x[0] - X).max())
    assert errs[1] < 2e-3
    assert 3.3 < errs[0] / errs[1] < 4.7


# ---------------------------------------------------------------- P3

def test_steady_state_satisfies_monge_ampere_config1():
    """Eq. (MA) at steady state: |Omega_c| rho det D^2 Psi = 1 after the
    normalisation, det > 0 and no inverted cell (Sect. 4.5 quality measure).
    Config 1 (33^2 ring, dt = 1e-4) reaches max|u_t| < 1e-6 uncapped."""
    prob = W.config1().replace(max_steps=20000)
    r = oracle.solve(prob)
    assert r.status == "ok" and r.residual <= 1e-6
    q = oracle.quality(prob, r.psi)
    assert abs(q["Emax"] - 1) < 2e-6 and abs(q["E2"] - 1) < 2e-6
    assert q["min_det"] > 0.1 and q["min_cell"] > 0
    # the residual decays (pseudo-time convergence, Sect. 4.4)
    assert np.all(np.diff(r.res[100:]) <= 1e-12)
    # the capped run stops at 2000 steps, not converged
    r2 = oracle.solve(W.config1())
    assert r2.status == "not_converged" and r2.steps == 2000 and r2.residual > 1e-6
    np.testing.assert_array_equal(r2.res, r.res[:2000])


# ---------------------------------------------------------------- P4

def test_separable_density_reduces_to_1d():
    """For rho = f(x) g(y) the LOG flow keeps v sum-separable on a single
    domain: the 2D mesh coordinates equal two independent 1D runs at every
    step.  (Under the parallel transmission of Eq. transmission_condition3
    the one-step lag of the Dirichlet data breaks exact separability by
    O(dt), so this pin is single-domain only.)"""
    fx, fy = (6.0, 60.0, 0.35), (3.0, 25.0, 0.7)
    mon2 = W.product_monitor([fx, fy])
    n = (29, 23, 1)
    dt = 0.05 * min(1 / 28 ** 2, 1 / 22 ** 2)
    p2 = W.Problem(dim=2, n=n, monitor=mon2, dt=dt, tol=0.0, max_steps=300)
    r2 = oracle.solve(p2)
    m1x = W.Monitor("sum", 1.0, [W.Term("bump", fx[0], fx[1], 0.0, (fx[2], 0, 0))])
    m1y = W.Monitor("sum", 1.0, [W.Term("bump", fy[0], fy[1], 0.0, (fy[2], 0, 0))])
    rx = oracle.solve(W.Problem(dim=1, n=(29, 1, 1), monitor=m1x, dt=dt, tol=0.0,
                                max_steps=300))
    ry = oracle.solve(W.Problem(dim=1, n=(23, 1, 1), monitor=m1y, dt=dt, tol=0.0,
                                max_steps=300))
    assert np.abs(r2.x[0] - _identity(p2)[0]).max() > 1e-2
    np.testing.assert_allclose(r2.x[0], np.broadcast_to(rx.x[0], (23, 29)), atol=1e-12)
    np.testing.assert_allclose(r2.x[1], np.broadcast_to(ry.x[0][:, None], (23, 29)),
                               atol=1e-12)
    # 3D, three factors
    mon3 = W.product_monitor([fx, fy, (4.0, 30.0, 0.5)])
    p3 = W.Problem(dim=3, n=(13, 11, 9), monitor=mon3, dt=0.03 / 144, tol=0.0, max_steps=80)
    r3 = oracle.solve(p3)
    mz = W.Monitor("sum", 1.0, [W.Term("bump", 4.0, 30.0, 0.0, (0.5, 0, 0))])
    rz = oracle.solve(W.Problem(dim=1, n=(9, 1, 1), monitor=mz, dt=0.03 / 144, tol=0.0,
                                max_steps=80))
    np.testing.assert_allclose(r3.x[2], np.broadcast_to(rz.x[0][:, None, None], (9, 11, 13)),
                               atol=1e-12)


def test_symmetric_density_gives_symmetric_mesh():
    """A ring centred in the square is invariant under the square's
    symmetries, so Psi is too -- on one domain and on a mirror-symmetric
    2x2 block decomposition (any index slip in the stencil, the mirror or
    the transmission breaks it)."""
    for parts, o in [((1, 1, 1), 0), ((2, 2, 1), 4)]:
        prob = W.Problem(dim=2, n=(26, 26, 1), monitor=W.ring_monitor(), parts=parts,
                         overlap=o, dt=W.dt_for((26, 26, 1), 2), tol=0.0, max_steps=300)
        r = oracle.solve(prob)
        xs = np.meshgrid(*_xi(prob), indexing="xy")
        v = r.psi - 0.5 * (xs[0] ** 2 + xs[1] ** 2)   # deviation potential
        np.testing.assert_allclose(v, v.T, atol=1e-13)
        np.testing.assert_allclose(v, v[::-1, :], atol=1e-13)
        np.testing.assert_allclose(v, v[:, ::-1], atol=1e-13)
        np.testing.assert_allclose(r.x[0][:, ::-1], 1.0 - r.x[0], atol=1e-13)
        assert np.abs(r.x[0] - _identity(prob)[0]).max() > 1e-3  # it did move


# ---------------------------------------------------------------- P5

@pytest.mark.parametrize("alternating", [0, 1])
def test_dd_steady_state_equals_single_domain(alternating):
    """Sect. 4.4 (steady-state study): the DD steady state converges to the
    single-domain one.  With the global normalisation the single-domain
    steady state is an exact fixed point of the DD step."""
    base = W.Problem(dim=2, n=(33, 33, 1), monitor=W.ring_monitor(), dt=1e-4, tol=1e-10,
                     max_steps=60000)
    sd = oracle.solve(base)
    dd = oracle.solve(base.replace(parts=(2, 2, 1), overlap=4, alternating=alternating))
    assert sd.status == "ok" and dd.status == "ok"
    assert np.abs(dd.x - sd.x).max() < 1e-7


def test_dd_error_decreases_with_overlap():
    """Sect. 4.4 overlap study (5, 9, 11, 15 points): after a fixed number of
    steps the DD-vs-SD error decreases as the overlap grows."""
    gold = json.load(open(os.path.join(GOLD, "convergence_slopes.json")))
    base = W.Problem(dim=2, n=(65, 65, 1), monitor=W.ring_monitor(),
                     dt=W.dt_for((65, 65, 1), 2), tol=0.0, max_steps=300)
    sd = oracle.solve(base)
    errs = []
    for o in [3] + gold["overlap_points"]:
        dd = oracle.solve(base.replace(parts=(2, 2, 1), overlap=o))
        errs.append(np.abs(dd.psi - sd.psi).max() / np.abs(sd.psi).max())
    assert all(a > b for a, b in zip(errs, errs[1:])), errs


# ---------------------------------------------------------------- P6

def test_time_convergence_first_order():
    """Sect. 4.4 forward-Euler study: DD (4 subdomains) vs a small-step
    single-domain reference at equal pseudo time; relative L1/L2/Linf errors
    fall with slope ~1 (paper: 1.01, 1.04, 1.03)."""
    gold = json.load(open(os.path.join(GOLD, "convergence_slopes.json")))
    n = 33
    h2 = (1.0 / (n - 1)) ** 2
    T = 100 * h2
    ref_c = gold["reference_time_step_over_hxi_heta"]
    ref = oracle.solve(W.Problem(dim=2, n=(n, n, 1), monitor=W.ring_monitor(), dt=T / round(T / (ref_c * h2)),
                                 tol=0.0, max_steps=int(round(T / (ref_c * h2)))))
    cs = gold["time_steps_over_hxi_heta"]
    e = []
    for c in cs:
        st = int(round(T / (c * h2)))
        dd = oracle.solve(W.Problem(dim=2, n=(n, n, 1), monitor=W.ring_monitor(), dt=T / st,
                                    tol=0.0, max_steps=st, parts=(2, 2, 1), overlap=3))
        d = dd.psi - ref.psi
        e.append([np.abs(d).sum() / np.abs(ref.psi).sum(),
                  math.sqrt((d * d).sum() / (ref.psi ** 2).sum()),
                  np.abs(d).max() / np.abs(ref.psi).max()])
    e = np.array(e)
    for k in range(3):
        slope = np.polyfit(np.log(cs), np.log(e[:, k]), 1)[0]
        assert 0.85 <= slope <= 1.2, slope


def test_space_convergence_second_order():
    """Sect. 4.4 space study: the DD steady-state mesh converges at second
    order in h (paper: slopes 1.85, 2.01, 1.99 in Linf, L1, L2).  Without a
    finer reference, the order follows from three nested grids: the
    differences 17->33 and 33->65 at the common nodes shrink by 2^p."""
    gold = json.load(open(os.path.join(GOLD, "convergence_slopes.json")))
    assert min(gold["space_slopes"].values()) > 1.7
    xs = {}
    for n in (17, 33, 65):
        prob = W.Problem(dim=2, n=(n, n, 1), monitor=W.ring_monitor(), parts=(2, 2, 1),
                         overlap=4, dt=W.dt_for((n, n, 1), 2), tol=1e-9, max_steps=10 ** 7)
        r = oracle.solve(prob)
        assert r.status == "ok"
        s = (n - 1) // 16
        xs[n] = r.x[:, ::s, ::s]
    d1, d2 = xs[17] - xs[33], xs[33] - xs[65]
    for norm in (lambda d: np.abs(d).sum(), lambda d: math.sqrt((d * d).sum()),
                 lambda d: np.abs(d).max()):
        order = math.log2(norm(d1) / norm(d2))
        assert 1.7 <= order <= 2.3, order


# ---------------------------------------------------------------- stop rule, variants

def test_stop_rule_and_status():
    prob = W.small_case(2, 17, steps=50)
    r = oracle.solve(prob.replace(tol=1e9, check_every=7))
    assert r.status == "ok" and r.steps == 7
    r = oracle.solve(prob.replace(tol=1e9))
    assert r.status == "ok" and r.steps == 1
    r = oracle.solve(prob)
    assert r.status == "not_converged" and r.steps == 50
    # a wildly unstable step tangles and reports it, with a finite mesh
    r = oracle.solve(prob.replace(dt=prob.dt * 40, max_steps=400))
    assert r.status == "tangled" and np.all(np.isfinite(r.x))
    # ANY (Algorithm 1 step 6: min over subdomains) never exceeds ALL (max)
    pdd = prob.replace(parts=(2, 2, 1), overlap=4, max_steps=40)
    ra = oracle.solve(pdd)
    rn = oracle.solve(pdd.replace(stop_rule="any"))
    assert np.all(rn.res <= ra.res) and np.any(rn.res < ra.res)
    # L2 increment norm (Eq. dd_stop_criterion) is O(dt) smaller than max|u_t|
    rl = oracle.solve(pdd.replace(stop_norm="l2_increment"))
    assert np.all(rl.res <= pdd.dt * ra.res * 1.0000001)


def test_root_form_has_the_same_steady_state():
    """The d-th-root right-hand side (|Omega_c| rho det / theta)^(1/d) - 1
    vanishes exactly where the log form does, so both flows share the
    steady state of Eq. (MA)."""
    base = W.Problem(dim=2, n=(21, 21, 1), monitor=W.ring_monitor(), dt=W.dt_for((21, 21, 1), 2),
                     tol=1e-10, max_steps=100000)
    a = oracle.solve(base)
    b = oracle.solve(base.replace(rhs="root"))
    c = oracle.solve(base.replace(rhs="root", lag_theta=1))
    assert a.status == b.status == c.status == "ok"
    assert np.abs(a.x - b.x).max() < 1e-7 and np.abs(a.x - c.x).max() < 1e-7


def test_warm_start_from_steady_state_is_stationary():
    """Sect. 2: at later physical times the flow restarts from the previous
    steady state; restarting from a converged Psi stops at once."""
    prob = W.config1().replace(max_steps=20000)
    r = oracle.solve(prob)
    r2 = oracle.solve(prob, psi0=r.psi)
    assert r2.status == "ok" and r2.steps == 1
    assert np.abs(r2.x - r.x).max() < 1e-9


def test_quality_measure_magnitude_matches_paper_table():
    """Sect. 4.5 / Table quality_measure_table, loosely: with J the
    determinant of the mesh Jacobian (centred differences of the computed
    mesh), E_2 of a converged single-domain mesh is within 1% of the printed
    values at 21^2 and 41^2 and falls with refinement.  The paper does not
    state the monitor, step or tolerances of that table; the Burgers-front
    arc-length monitor of Eq. (test_fn1) is used here."""
    gold = json.load(open(os.path.join(GOLD, "quality_table.json")))["rows"]["whole domain"]
    e2s = []
    for n in (21, 41):
        mon = W.Monitor("arclen_burgers", 1.0, [], p0=0.01)
        prob = W.Problem(dim=2, n=(n, n, 1), monitor=mon, dt=W.dt_for((n, n, 1), 2, cfl=0.02),
                         tol=1e-6, max_steps=10 ** 6)
        r = oracle.solve(prob)
        assert r.status == "ok"
        X, Y = r.x
        h = 1.0 / (n - 1)
        J = (np.gradient(X, h, axis=1) * np.gradient(Y, h, axis=0) -
             np.gradient(X, h, axis=0) * np.gradient(Y, h, axis=1))
        rho = oracle.monitor_eval(mon, 2, np.stack([X.ravel(), Y.ravel()], 1)).reshape(X.shape)
        w = np.full((n, n), h * h)
        w[[0, -1], :] *= 0.5
        w[:, [0, -1]] *= 0.5
        E = rho * J / (w * rho * J).sum()
        e2 = math.sqrt((w * E * E).sum() / w.sum())
        e2s.append(e2)
        assert abs(e2 - gold[str(n)]["E2"]) < 0.01
    assert e2s[1] < e2s[0]


# ------------------------------------------------------------------ tabulated density

def _table_monitor(values, tlo, thi):
    return W.Monitor(kind="table", table=np.asarray(values, dtype=np.float64),
                     tlo=tuple(tlo) + (0.0,) * (3 - len(tlo)),
                     thi=tuple(thi) + (1.0,) * (3 - len(thi)))


def test_table_monitor_is_exact_on_multilinear_densities():
    """Multilinear interpolation reproduces a multilinear density exactly
    (inside the box), and outside it takes the value at the clamped point."""
    rng = np.random.default_rng(5)
    # 2D: rho = 2 + x + 3y + 0.5 x y on a 7 x 9 table over [-0.1, 1.2] x [0, 1.1]
    f2 = lambda x, y: 2.0 + x + 3.0 * y + 0.5 * x * y
    xs, ys = np.linspace(-0.1, 1.2, 7), np.linspace(0.0, 1.1, 9)
    tab = f2(xs[None, :], ys[:, None])
    mon = _table_monitor(tab, (-0.1, 0.0), (1.2, 1.1))
    pts = rng.uniform([-0.1, 0.0], [1.2, 1.1], size=(200, 2))
    got = oracle.monitor_eval(mon, 2, pts)
    assert np.abs(got - f2(pts[:, 0], pts[:, 1])).max() < 1e-13
    out = np.array([[-0.5, 0.3], [1.7, 2.0], [0.4, -1.0]])
    clamped = np.clip(out, [-0.1, 0.0], [1.2, 1.1])
    assert np.abs(oracle.monitor_eval(mon, 2, out) - f2(clamped[:, 0], clamped[:, 1])).max() < 1e-13
    # 3D: a trilinear density on a 5 x 4 x 6 table
    f3 = lambda x, y, z: 1 + x + 2 * y + 3 * z + x * y + y * z + x * z + x * y * z
    gx, gy, gz = np.linspace(0, 1, 5), np.linspace(0, 1, 4), np.linspace(0, 1, 6)
    tab3 = f3(gx[None, None, :], gy[None, :, None], gz[:, None, None])
    mon3 = _table_monitor(tab3, (0, 0, 0), (1, 1, 1))
    pts3 = rng.uniform(0, 1, size=(200, 3))
    got3 = oracle.monitor_eval(mon3, 3, pts3)
    assert np.abs(got3 - f3(pts3[:, 0], pts3[:, 1], pts3[:, 2])).max() < 1e-13


def test_table_monitor_matches_scipy_linear_interpolation():
    """A random positive table against scipy's regular-grid linear
    interpolator (an independent library routine)."""
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(6)
    for dim, shape in ((2, (11, 8)), (3, (5, 7, 6))):
        tab = rng.uniform(0.5, 3.0, size=shape)            # (n_z, n_y, n_x) order
        lo, hi = rng.uniform(-1, 0, size=dim), rng.uniform(1, 2, size=dim)
        axes = [np.linspace(lo[a], hi[a], shape[::-1][a]) for a in range(dim)]
        f = interp.RegularGridInterpolator(axes, np.transpose(tab), method="linear")
        pts = rng.uniform(lo, hi, size=(300, dim))
        got = oracle.monitor_eval(_table_monitor(tab, lo, hi), dim, pts)
        assert np.abs(got - f(pts)).max() < 1e-13


def test_tabulated_ring_converges_to_the_analytic_ring():
    """The mesh of a ring density sampled on finer and finer tables tends to
    the mesh of the analytic ring at second order in the table spacing."""
    base = W.Problem(dim=2, n=(33, 33, 1), monitor=W.ring_monitor(), dt=W.dt_for((33, 33, 1), 2),
                     tol=0.0, max_steps=150)
    ref = oracle.solve(base).x
    errs = []
    for nt in (33, 65, 129):
        g = np.linspace(0.0, 1.0, nt)
        X, Y = np.meshgrid(g, g, indexing="xy")
        vals = oracle.monitor_eval(W.ring_monitor(), 2, np.stack([X.ravel(), Y.ravel()], 1))
        mon = _table_monitor(vals.reshape(nt, nt), (0, 0), (1, 1))
        errs.append(np.abs(oracle.solve(base.replace(monitor=mon)).x - ref).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert errs[2] < errs[1] < errs[0]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, (errs, r1, r2)


# ------------------------------------------------------------------ one step in closed form

def _rho_np(mon, pts):
    """Sum-of-terms density at points (n, dim) from the term shapes, numpy."""
    r = np.full(pts.shape[0], float(mon.base))
    for t in mon.terms:
        q = ((pts - np.asarray(t.c[: pts.shape[1]])) ** 2).sum(1)
        if t.type == "bump":
            r += t.amp * np.exp(-t.width * q)
        elif t.type == "ring":
            r += t.amp * np.exp(-t.width * (q - t.r2) ** 2)
        else:
            raise ValueError(t.type)
    return r


def _trapezoid(prob):
    """Trapezoid weights on the global grid, arrays (z, y, x)."""
    ws = []
    for a in range(prob.dim):
        h = (prob.hi[a] - prob.lo[a]) / (prob.n[a] - 1)
        w = np.full(prob.n[a], h)
        w[[0, -1]] *= 0.5
        ws.append(w)
    W_ = ws[0]
    for a in range(1, prob.dim):
        W_ = np.multiply.outer(ws[a], W_)   # later axes are slower
    return W_


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("rhs", ["log", "root"])
def test_first_step_from_identity_in_closed_form(dim, rhs):
    """From Psi^0 = |xi|^2/2 (Eq. incond) the mesh is the identity and
    D^2 Psi = I at every node, so one forward-Euler step of Eq. (pmae) moves
    Psi by dt log(|Omega_c| rho(xi)/theta) exactly, and the root form by
    dt ((|Omega_c| rho(xi)/theta)^(1/d) - 1), with theta the trapezoid sum of
    rho over the nodes (the normalisation of Eq. edp).  Single domain and
    blocks alike: the transmission does not enter the first step."""
    n = {1: 17, 2: 11, 3: 7}[dim]
    lo, hi = (0.1, -0.2, 0.3), (1.2, 0.7, 1.1)
    mon = W.Monitor("sum", 1.0, [W.Term("bump", 7.0, 9.0, 0.0, (0.5, 0.3, 0.6)),
                                  W.Term("ring", 3.0, 20.0, 0.1, (0.7, 0.2, 0.8))])
    nn = (n, n if dim > 1 else 1, n if dim > 2 else 1)
    parts = {1: (2, 1, 1), 2: (2, 2, 1), 3: (2, 1, 2)}[dim]
    for pr, o in (((1, 1, 1), 0), (parts, 3)):
        prob = W.Problem(dim=dim, n=nn, lo=lo, hi=hi, monitor=mon, parts=pr, overlap=o,
                         dt=1e-3, tol=0.0, max_steps=1, rhs=rhs)
        r = oracle.solve(prob)
        X = np.stack([g.T for g in np.meshgrid(*_xi(prob), indexing="ij")])
        pts = X.reshape(dim, -1).T
        rho = _rho_np(mon, pts).reshape(X.shape[1:])
        vol = np.prod([hi[a] - lo[a] for a in range(dim)])
        theta = (_trapezoid(prob) * rho).sum()
        z = vol * rho / theta
        F = np.log(z) if rhs == "log" else z ** (1.0 / dim) - 1.0
        psi0 = 0.5 * (X ** 2).sum(0)
        np.testing.assert_allclose(r.psi - psi0, 1e-3 * F, rtol=0, atol=1e-15)
        assert abs(r.theta - theta) < 1e-12 * theta


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_l2_increment_residual_is_the_trapezoid_norm_of_the_step(dim):
    """Eq. (dd_stop_criterion): on one domain the L2 residual of step k is
    (sum_nodes w (Psi^{k+1} - Psi^k)^2)^(1/2) with the trapezoid weights of
    Omega_c, taken here from two runs stopped after k and k + 1 steps."""
    n = {1: 33, 2: 17, 3: 9}[dim]
    prob = W.small_case(dim, n, steps=6).replace(stop_norm="l2_increment")
    w = _trapezoid(prob)
    for k in (0, 3, 5):
        a = oracle.solve(prob.replace(max_steps=k)) if k else None
        b = oracle.solve(prob.replace(max_steps=k + 1))
        if a is None:
            X = np.stack([g.T for g in np.meshgrid(*_xi(prob), indexing="ij")])
            psi_k = 0.5 * (X ** 2).sum(0)
        else:
            psi_k = a.psi
        want = math.sqrt((w * (b.psi - psi_k) ** 2).sum())
        assert want > 0
        assert abs(b.res[k] - want) <= 1e-9 * want, (k, b.res[k], want)


def test_alternating_transmission_takes_new_values_from_preceding_owners_only():
    """Algorithm 1 on two slabs: subdomain 1 takes subdomain 2's values of
    the previous step (as in the parallel form, Eq. transmission_condition1)
    and subdomain 2 takes subdomain 1's new values (Eq.
    transmission_condition2).  From the identity the two forms agree after
    one step; later (three steps: with overlap 4 a transmission value reaches
    the neighbour's core after two more), the nodes owned by subdomain 1
    still agree with the parallel run exactly, and only subdomain 2 differs.
    (Without the global normalisation, as the subdomain equations of Eq.
    pmae1a are printed: theta couples every node and would shift Psi
    everywhere by a constant.)"""
    base = W.Problem(dim=2, n=(21, 13, 1), monitor=W.ring_monitor(), parts=(2, 1, 1),
                     overlap=4, dt=W.dt_for((21, 13, 1), 2), tol=0.0, max_steps=1,
                     normalize="none")
    _, _, clo, chi = oracle.extents(21, 2, 4)
    for steps in (1, 3):
        par = oracle.solve(base.replace(max_steps=steps))
        alt = oracle.solve(base.replace(max_steps=steps, alternating=1))
        own1 = (slice(None), slice(clo[0], chi[0] + 1))
        own2 = (slice(None), slice(clo[1], chi[1] + 1))
        np.testing.assert_array_equal(alt.psi[own1], par.psi[own1])
        if steps == 1:
            np.testing.assert_array_equal(alt.psi, par.psi)
        else:
            assert np.abs(alt.psi[own2] - par.psi[own2]).max() > 1e-9


# ------------------------------------------------------------------ frozen interface data

def test_exchange_every_one_is_the_parallel_method():
    """K = 1 exchanges the interface data at every step: bitwise the same
    run as the parallel form of Eq. (transmission_condition3)."""
    prob = W.small_case(2, 25, parts=(2, 2, 1), overlap=4, steps=40)
    a = oracle.solve(prob)
    b = oracle.solve(prob.replace(exchange_every=1))
    c = oracle.solve(prob.replace(exchange_every=0))
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.x, c.x)
    np.testing.assert_array_equal(a.res, b.res)


def test_frozen_interface_data_lag_grows_with_the_interval_and_vanishes_at_steady_state():
    """Interface data frozen over intervals of K steps (Sect. 3: each
    subdomain is integrated over Delta tau with its neighbours' data of the
    interval's start).  At a fixed pseudo time the DD mesh departs further
    from the single-domain mesh as K grows; the steady state, a fixed point
    of every exchange schedule under the global normalisation, is the
    single-domain steady state for every K."""
    base = W.Problem(dim=2, n=(33, 33, 1), monitor=W.ring_monitor(), dt=1e-4, tol=0.0,
                     max_steps=400)
    sd = oracle.solve(base)
    errs = []
    for K in (1, 2, 4, 8):
        dd = oracle.solve(base.replace(parts=(2, 2, 1), overlap=4, exchange_every=K))
        errs.append(np.abs(dd.x - sd.x).max())
    assert all(a < b for a, b in zip(errs, errs[1:])), errs
    steady = base.replace(tol=1e-10, max_steps=60000)
    ref = oracle.solve(steady)
    for K in (2, 8):
        dd = oracle.solve(steady.replace(parts=(2, 2, 1), overlap=4, exchange_every=K,
                                         check_every=K))
        assert dd.status == "ok" and np.abs(dd.x - ref.x).max() < 1e-7


def test_frozen_interface_data_hold_between_exchanges():
    """Between exchanges a subdomain sees constant Dirichlet data.  With
    K = 5 the first exchange after step 0 is at step 5 (it writes the
    Dirichlet values of Psi^6), so up to that point the run equals the one
    with K = 10; the new data reach the owned cores (two nodes inside the
    Dirichlet layer at overlap 4) two steps later, at Psi^8.  Unnormalised
    subdomain equations (Eq. pmae1a), so that no global constant couples the
    subdomains."""
    prob = W.small_case(2, 25, parts=(2, 2, 1), overlap=4, steps=8).replace(normalize="none")
    for steps in range(1, 9):
        a = oracle.solve(prob.replace(max_steps=steps, exchange_every=5))
        b = oracle.solve(prob.replace(max_steps=steps, exchange_every=10))
        if steps <= 7:
            np.testing.assert_array_equal(a.psi, b.psi)
        else:
            assert np.abs(a.psi - b.psi).max() > 0


def test_owner_stencil_determinant_output():
    """The oracle's det output is det D_h^2 Psi at each global node from its
    owner's stencil: on one domain it equals the operator applied to the
    combined Psi everywhere; on blocks, wherever a node's 3 x 3 stencil lies
    in its owner's core (so the combined Psi holds the owner's values)."""
    single = W.small_case(2, 23, steps=40)
    r = oracle.solve(single, want_det=True)
    xs = np.meshgrid(*_xi(single), indexing="xy")
    v = r.psi - 0.5 * (xs[0] ** 2 + xs[1] ** 2)
    _, det, _, _ = oracle.operator(single, v)
    np.testing.assert_allclose(r.det, det, rtol=0, atol=1e-12)
    dd = single.replace(parts=(2, 2, 1), overlap=4)
    r = oracle.solve(dd, want_det=True)
    v = r.psi - 0.5 * (xs[0] ** 2 + xs[1] ** 2)
    _, det, _, _ = oracle.operator(dd, v)
    _, _, clo, chi = oracle.extents(23, 2, 4)
    own = np.searchsorted(chi, np.arange(23))          # core index per axis
    same = np.ones((23, 23), dtype=bool)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            jj = np.clip(np.arange(23) + dj, 0, 22)
            ii = np.clip(np.arange(23) + di, 0, 22)
            same &= (own[jj][:, None] == own[:, None]) & (own[ii][None, :] == own[None, :])
    assert same.sum() > 300 and (~same).sum() > 50
    np.testing.assert_allclose(r.det[same], det[same], rtol=0, atol=1e-12)
    assert np.abs(r.det - det).max() > 1e-9   # the overlap copies do differ
