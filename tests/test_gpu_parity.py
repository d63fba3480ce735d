"""Parity of the sm_103a path (through the C ABI) with the FP64 oracle.

FP64 device runs must match node positions within 1e-11 (times the domain
size); FP32 runs within 1e-5, after the same number of steps.  Step counts,
statuses and the stop decision must agree exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2006_14602_gb300 import pma
from paper_2006_14602_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()


def _size(prob):
    return max(prob.hi[a] - prob.lo[a] for a in range(prob.dim))


def _check(prob, ref=None, tol=None, psi=True, **opts):
    if ref is None:
        ref = oracle.solve(prob)
    x, p, info = pma.solve(prob, want_psi=psi, **opts)
    if tol is None:
        tol = TOL64 if prob.precision == "fp64" else TOL32
    assert info.steps == ref.steps, (info.steps, ref.steps)
    assert pma.STATUS_NAMES[info.status] == ref.status
    err = np.abs(x - ref.x).max() / _size(prob)
    assert err <= tol, err
    if psi and prob.precision == "fp64":
        assert np.abs(p - ref.psi).max() <= 1e3 * tol, np.abs(p - ref.psi).max()
    return x, p, info, ref, err


# ------------------------------------------------------------------ 2D

def test_config1_fp64():
    """33^2 ring, dt = 1e-4, 2000-step cap (not converged at the cap)."""
    prob = W.config1()
    x, p, info, ref, err = _check(prob)
    assert info.status == pma.PMA_NOT_CONVERGED
    assert abs(info.residual - ref.residual) <= 1e-9 * ref.residual


def test_config1_uncapped_converges_at_same_step():
    prob = W.config1().replace(max_steps=6000)
    x, p, info, ref, err = _check(prob)
    assert info.status == pma.PMA_OK and info.steps == ref.steps == 2857


@pytest.mark.parametrize("resident", [0, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,parts,o", [((45, 37), (3, 2), 5), ((70, 33), (1, 3), 4),
                                       ((21, 64), (2, 1), 2), ((97, 65), (4, 3), 8)])
def test_dd_2d_ragged(prec, n, parts, o, resident):
    prob = W.Problem(dim=2, n=(n[0], n[1], 1), monitor=W.ring_monitor(), parts=(parts[0], parts[1], 1),
                     overlap=o, dt=W.dt_for((n[0], n[1], 1), 2), tol=0.0, max_steps=150,
                     precision=prec)
    _check(prob, resident=resident, window_steps=40)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_subdomains_wider_than_one_band(prec):
    """Subdomains of about 1150 columns are cut into two strips of bands
    (at most 1024 columns each): transmission columns, mirror halos and the
    strip seam all meet in one request."""
    n = (2300, 40, 1)
    prob = W.Problem(dim=2, n=n, monitor=W.sine_monitor(), parts=(2, 1, 1), overlap=6,
                     dt=W.dt_for(n, 2), tol=0.0, max_steps=25, precision=prec)
    _check(prob, psi=False)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,parts,o", [((123, 201), (1, 1), 0), ((150, 400), (2, 2), 6)])
def test_tma_staged_bands_ragged(prec, n, parts, o):
    """Subdomains of several bands staged by TMA boxes: the last band of a
    subdomain is shorter than its box (rows beyond it or outside the buffer
    are fetched and ignored), mirror rows come from inside the box on
    physical faces, transmission rows and columns on inner ones."""
    prob = W.Problem(dim=2, n=(n[0], n[1], 1), monitor=W.ring_monitor(), parts=(parts[0], parts[1], 1),
                     overlap=o, dt=W.dt_for((n[0], n[1], 1), 2), tol=0.0, max_steps=40,
                     precision=prec)
    _check(prob, psi=False)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,parts,o", [(2, (3, 41, 1), (1, 2, 1), 2), (2, (41, 3, 1), (2, 1, 1), 2),
                                           (2, (3, 3, 1), (1, 1, 1), 0), (3, (3, 3, 3), (1, 1, 1), 0),
                                           (3, (5, 4, 3), (1, 1, 1), 0), (3, (3, 17, 9), (1, 2, 1), 2)])
def test_degenerate_minimum_grids(prec, dim, n, parts, o):
    """The smallest grids the method allows (3 nodes on an axis, the
    thinnest decompositions): runs of 4 nodes padded past the grid, boxes of
    a few columns, every node on a physical or transmission face."""
    prob = W.Problem(dim=dim, n=n, monitor=W.ring_monitor(dim) if dim == 2 else W.shell_monitor(),
                     parts=parts, overlap=o, dt=W.dt_for(n, dim, cfl=0.1 if dim == 2 else 0.05),
                     tol=0.0, max_steps=20, precision=prec)
    _check(prob, psi=False)


@pytest.mark.parametrize("mon", ["sine", "bumps", "product", "burgers"])
def test_monitor_kinds_2d(mon):
    rng = np.random.default_rng(5)
    m = {"sine": W.sine_monitor(), "bumps": W.random_bumps(rng, 2, 4),
         "product": W.product_monitor([(4.0, 40.0, 0.3), (2.0, 20.0, 0.6)]),
         "burgers": W.Monitor("arclen_burgers", 1.0, [], p0=0.05)}[mon]
    prob = W.Problem(dim=2, n=(41, 39, 1), monitor=m, parts=(2, 2, 1), overlap=4,
                     dt=W.dt_for((41, 39, 1), 2, cfl=0.03), tol=0.0, max_steps=100,
                     precision="fp64")
    _check(prob)


def test_spiral_monitor_short():
    prob = W.Problem(dim=2, n=(33, 33, 1), monitor=W.Monitor("arclen_spiral", 1.0, []),
                     dt=W.dt_for((33, 33, 1), 2, cfl=0.001), tol=0.0, max_steps=20,
                     precision="fp64")
    _check(prob)


@pytest.mark.parametrize("variant", ["l2", "any", "check7", "none", "root", "root_none"])
def test_stop_rules_and_variants(variant):
    base = W.Problem(dim=2, n=(29, 29, 1), monitor=W.ring_monitor(), parts=(2, 2, 1), overlap=4,
                     dt=W.dt_for((29, 29, 1), 2), tol=2e-4, max_steps=3000, precision="fp64")
    prob = {"l2": base.replace(stop_norm="l2_increment", tol=1e-9),
            "any": base.replace(stop_rule="any"),
            "check7": base.replace(check_every=7),
            "none": base.replace(normalize="none", tol=0.0, max_steps=200),
            "root": base.replace(rhs="root", lag_theta=1),
            # the root form of the unnormalised subdomain equations:
            # (rho det)^(1/d) - 1
            "root_none": base.replace(rhs="root", lag_theta=1, normalize="none", tol=0.0,
                                      max_steps=200)}[variant]
    x, p, info, ref, err = _check(prob)
    if variant not in ("none", "root_none"):
        assert info.status == pma.PMA_OK
    assert abs(info.residual - ref.residual) <= 1e-8 * max(ref.residual, 1e-300)


def test_warm_start():
    prob = W.config1().replace(max_steps=300)
    first = oracle.solve(prob)
    ref = oracle.solve(prob, psi0=first.psi)
    x, p, info = pma.solve(prob, psi0=first.psi)
    assert info.steps == ref.steps
    assert np.abs(x - ref.x).max() <= TOL64


def test_resume_from_the_returned_psi():
    """Checkpoint / resume through the warm start of Sect. 2: on one domain
    the combined Psi after n steps is the whole state, so n steps, then m
    more from the returned Psi, give the mesh of one n + m-step run.  On
    blocks the restart also resets the transmission nodes to their owners'
    current values (the uninterrupted parallel run holds the previous
    ones), exactly as the oracle's restart does."""
    one = W.Problem(dim=2, n=(41, 37, 1), monitor=W.ring_monitor(), dt=W.dt_for((41, 37, 1), 2),
                    tol=0.0, max_steps=300, precision="fp64")
    for prob in (one, one.replace(parts=(2, 2, 1), overlap=4)):
        _, psi, _ = pma.solve(prob)
        x2, _, i2 = pma.solve(prob.replace(max_steps=200), psi0=psi)
        assert i2.steps == 200
        ref = oracle.solve(prob.replace(max_steps=200), psi0=oracle.solve(prob).psi)
        assert np.abs(x2 - ref.x).max() <= TOL64
        if prob.parts == (1, 1, 1):
            x, _, _ = pma.solve(prob.replace(max_steps=500))
            assert np.abs(x2 - x).max() <= TOL64


def test_tangle_is_reported_with_last_valid_mesh():
    prob = W.small_case(2, 25, parts=(2, 2, 1), overlap=4, steps=400).replace(
        dt=W.dt_for((25, 25, 1), 2, cfl=4.0))
    ref = oracle.solve(prob)
    assert ref.status == "tangled"
    x, p, info = pma.solve(prob)
    assert info.status == pma.PMA_ERR_TANGLED and info.steps == ref.steps
    assert np.abs(x - ref.x).max() <= 1e-9
    assert info.min_det <= 0 or not np.isfinite(info.min_det)


def test_uniform_and_zero_steps():
    prob = W.Problem(dim=2, n=(30, 30, 1), monitor=W.uniform_monitor(2.0), parts=(2, 2, 1),
                     overlap=4, dt=1e-4, tol=0.0, max_steps=100, precision="fp32")
    x, p, info = pma.solve(prob)
    ident = np.stack(np.meshgrid(np.linspace(0, 1, 30), np.linspace(0, 1, 30), indexing="xy"))
    assert np.abs(x - ident).max() < 1e-6
    x, p, info = pma.solve(prob.replace(max_steps=0))
    assert info.steps == 0 and info.status == pma.PMA_NOT_CONVERGED
    assert np.abs(x - ident).max() == 0.0


# ------------------------------------------------------------------ 3D

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,parts,o", [((19, 17, 15), (2, 2, 2), 4), ((26, 20, 35), (1, 2, 3), 5),
                                       ((40, 9, 11), (3, 1, 1), 3)])
def test_dd_3d(prec, n, parts, o):
    prob = W.Problem(dim=3, n=n, monitor=W.shell_monitor(), parts=parts, overlap=o,
                     dt=W.dt_for(n, 3, cfl=0.05), tol=0.0, max_steps=60, precision=prec)
    _check(prob)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tma_staged_boxes_all_extents(prec):
    """3D boxes of four extents in one subdomain (full / last rows x full /
    last planes, one pair of tensor maps each), mirror rows and planes on
    the physical faces."""
    n = (30, 44, 27)
    prob = W.Problem(dim=3, n=n, monitor=W.shell_monitor(), parts=(1, 2, 2), overlap=4,
                     dt=W.dt_for(n, 3, cfl=0.05), tol=0.0, max_steps=30, precision=prec)
    _check(prob, psi=False)


@pytest.mark.parametrize("mon", ["tanh_sphere", "nine_spheres"])
def test_monitor_kinds_3d(mon):
    kind = "arclen_" + mon
    lim = 1.0 if mon == "tanh_sphere" else 2.0
    prob = W.Problem(dim=3, n=(17, 17, 17), lo=(-lim,) * 3, hi=(lim,) * 3,
                     monitor=W.Monitor(kind, 1.0, []), parts=(2, 2, 2), overlap=4,
                     dt=W.dt_for((17, 17, 17), 3, (-lim,) * 3, (lim,) * 3, cfl=0.002),
                     tol=0.0, max_steps=15, precision="fp64")
    _check(prob)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,parts,o", [(2, (45, 37, 1), (3, 2, 1), 5),
                                           (2, (21, 40, 1), (2, 3, 1), 2),
                                           (3, (19, 17, 15), (2, 2, 2), 4),
                                           (3, (16, 24, 18), (1, 3, 2), 2)])
def test_alternating_transmission(prec, dim, n, parts, o):
    """Algorithm 1's alternating form: a transmission node whose owner
    precedes its subdomain takes the owner's new value.  Overlap 2 puts
    transmission nodes next to owned nodes, so the combination reads them
    too."""
    cfl = 0.1 if dim == 2 else 0.05
    mon = W.ring_monitor() if dim == 2 else W.shell_monitor()
    prob = W.Problem(dim=dim, n=n, monitor=mon, parts=parts, overlap=o, alternating=1,
                     dt=W.dt_for(n, dim, cfl=cfl), tol=0.0, max_steps=90 if dim == 2 else 40,
                     precision=prec)
    ref = oracle.solve(prob)
    par = oracle.solve(prob.replace(alternating=0))
    # the two transmission forms really differ on this problem
    assert np.abs(ref.x - par.x).max() > 1e-9
    _check(prob, ref)


def test_alternating_converges_at_the_oracle_step():
    prob = W.Problem(dim=2, n=(33, 33, 1), monitor=W.ring_monitor(), parts=(2, 2, 1), overlap=4,
                     alternating=1, dt=1e-4, tol=1e-6, max_steps=6000, precision="fp64")
    x, p, info, ref, err = _check(prob)
    assert info.status == pma.PMA_OK


def _sampled(mon, dim, nt, lo=0.0, hi=1.0):
    """The density `mon` sampled by the oracle on an nt^dim table."""
    g = np.linspace(lo, hi, nt)
    grids = np.meshgrid(*([g] * dim), indexing="ij")[::-1]  # x fastest
    pts = np.stack([q.ravel() for q in grids], 1)
    vals = oracle.monitor_eval(mon, dim, pts).reshape((nt,) * dim)
    return W.Monitor(kind="table", table=vals, tlo=(lo,) * 3, thi=(hi,) * 3)


@pytest.mark.parametrize("resident", [0, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tabulated_density_2d(prec, resident):
    """A density given as a table (sampled from the ring on a 97^2 grid,
    coarser than nothing else in the problem) through the same path."""
    mon = _sampled(W.ring_monitor(), 2, 97)
    prob = W.Problem(dim=2, n=(45, 37, 1), monitor=mon, parts=(3, 2, 1), overlap=5,
                     dt=W.dt_for((45, 37, 1), 2), tol=0.0, max_steps=120, precision=prec)
    _check(prob, resident=resident)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tabulated_density_3d(prec):
    mon = _sampled(W.shell_monitor(), 3, 25)
    prob = W.Problem(dim=3, n=(19, 17, 15), monitor=mon, parts=(2, 2, 2), overlap=4,
                     dt=W.dt_for((19, 17, 15), 3, cfl=0.05), tol=0.0, max_steps=40,
                     precision=prec)
    _check(prob)


def test_tabulated_density_is_validated():
    bad = np.ones((9, 9))
    bad[3, 4] = 0.0
    prob = W.Problem(dim=2, n=(21, 21, 1), monitor=W.Monitor(kind="table", table=bad),
                     dt=1e-4, tol=0.0, max_steps=5)
    with pytest.raises(pma.PmaError) as e:
        pma.solve(prob)
    assert e.value.status == pma.PMA_ERR_INVALID and "table" in pma.pma_last_error()


# ------------------------------------------------------------------ modes

def test_launch_modes_are_bitwise_identical():
    prob = W.Problem(dim=2, n=(50, 44, 1), monitor=W.ring_monitor(), parts=(3, 2, 1), overlap=6,
                     dt=W.dt_for((50, 44, 1), 2), tol=0.0, max_steps=77, precision="fp32")
    a = pma.solve(prob, window_steps=32, resident=0)[0]
    b = pma.solve(prob, window_steps=5, use_graphs=0, resident=0)[0]
    c = pma.solve(prob, launch_mode=pma.PMA_LAUNCH_PER_SUBDOMAIN, window_steps=16)[0]
    assert np.array_equal(a, b) and np.array_equal(a, c)
    # the resident path does not depend on the window either
    r1 = pma.solve(prob, window_steps=32, resident=4)[0]
    r2 = pma.solve(prob, window_steps=3, resident=4)[0]
    r3 = pma.solve(prob, window_steps=8, resident=4, resident_steps=50)[0]
    assert np.array_equal(r1, r2) and np.array_equal(r1, r3)
    # another tile shape, or the resident path, changes the summation order
    # of theta (a uniform offset of v), so positions agree to rounding
    ref = oracle.solve(prob)
    assert np.abs(r1 - a).max() < 1e-6 and np.abs(r1 - ref.x).max() < TOL32
    for t in range(4):
        d = pma.solve(prob, tile_2d=t, resident=0)[0]
        assert np.abs(d - a).max() < 1e-6 and np.abs(d - ref.x).max() < TOL32


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("variant", ["ragged", "l2_any", "tangle", "warm"])
def test_band_and_resident_paths_both_match_the_oracle(prec, variant):
    """The 2D band kernels (resident path off) and the cluster-resident path
    against the oracle on the same problem; the resident path really ran."""
    if variant == "ragged":
        prob = W.Problem(dim=2, n=(61, 47, 1), monitor=W.sine_monitor(), parts=(4, 3, 1),
                         overlap=5, dt=W.dt_for((61, 47, 1), 2), tol=0.0, max_steps=140,
                         precision=prec)
    elif variant == "l2_any":
        # the per-subdomain L2 increments combined by ANY (no stop: the
        # residual itself is compared)
        prob = W.Problem(dim=2, n=(40, 52, 1), monitor=W.ring_monitor(), parts=(2, 3, 1),
                         overlap=6, dt=W.dt_for((40, 52, 1), 2), tol=0.0, max_steps=150,
                         precision=prec, stop_norm="l2_increment", stop_rule="any")
    elif variant == "tangle":
        prob = W.small_case(2, 25, parts=(2, 2, 1), overlap=4, steps=400, precision=prec).replace(
            dt=W.dt_for((25, 25, 1), 2, cfl=4.0))
    else:
        prob = W.Problem(dim=2, n=(37, 41, 1), monitor=W.ring_monitor(), parts=(2, 2, 1),
                         overlap=4, dt=W.dt_for((37, 41, 1), 2), tol=0.0, max_steps=60,
                         precision=prec)
    psi0 = None
    if variant == "warm":
        psi0 = oracle.solve(prob.replace(max_steps=40, precision="fp64")).psi
    ref = oracle.solve(prob, psi0)
    tol = TOL64 if prec == "fp64" else TOL32
    if variant == "tangle":
        tol = max(tol, 1e-9)
    for resident in (0, 4):
        with pma.Context(0, resident=resident, window_steps=16) as ctx:
            rid = ctx.submit(prob, psi0)
            ctx.run()
            x, _, info = ctx.mesh(prob, rid)
            _, stats = pma.pma_get_stats(ctx.h)
        assert (stats.res_launches > 0) == bool(resident)
        assert info.steps == ref.steps and pma.STATUS_NAMES[info.status] == ref.status
        assert np.abs(x - ref.x).max() / _size(prob) <= tol, (resident, np.abs(x - ref.x).max())
        if variant == "l2_any":
            rel = 1e-8 if prec == "fp64" else 1e-3
            assert abs(info.residual - ref.residual) <= rel * ref.residual


def test_resident_and_band_agree_on_an_uneven_batch():
    """48 requests of the uneven batch (1-16 subdomains, odd and even
    overlaps, every resident class) over several windows: the resident path
    and the band kernels take the same number of steps with the same status
    and the same meshes to rounding; a sample of requests against the
    oracle."""
    probs = [p.replace(max_steps=200) for p in W.config4(count=48)]
    for prec in ("fp64", "fp32"):
        ps = [p.replace(precision=prec) for p in probs]
        res = pma.solve_many(ps, window_steps=16, resident=4)
        band = pma.solve_many(ps, window_steps=16, resident=0)
        for p, (xr, _, ir), (xb, _, ib) in zip(ps, res, band):
            assert (ir.steps, ir.status) == (ib.steps, ib.status), (p.n, p.parts)
            tol = 1e-9 if prec == "fp64" else 1e-4
            assert np.abs(xr - xb).max() / _size(p) <= tol, (p.n, p.parts)
    for k in (12, 17, 21):
        ref = oracle.solve(probs[k].replace(precision="fp64"))
        x, _, info = pma.solve(probs[k].replace(precision="fp64"), want_psi=False,
                               window_steps=16, resident=4)
        assert info.steps == ref.steps and pma.STATUS_NAMES[info.status] == ref.status
        assert np.abs(x - ref.x).max() / _size(probs[k]) <= TOL64


def test_resident_clusters_of_sixteen_and_packing():
    """Requests with 16, 9, 5, 2 and 1 subdomains packed into clusters of
    16 CTAs; each mesh bitwise equal to the request solved alone."""
    probs = []
    for parts, n in (((4, 4, 1), 96), ((3, 3, 1), 70), ((5, 1, 1), 90), ((1, 2, 1), 40),
                     ((1, 1, 1), 30), ((2, 2, 1), 50)):
        nn = (n, n - 7, 1)
        probs.append(W.Problem(dim=2, n=nn, monitor=W.ring_monitor(), parts=parts,
                               overlap=4 if parts != (1, 1, 1) else 0, dt=W.dt_for(nn, 2),
                               tol=0.0, max_steps=90, precision="fp32"))
    mixed = pma.solve_many(probs, window_steps=20, resident=4)
    for p, m in zip(probs, mixed):
        alone = pma.solve(p, want_psi=False, resident=4)
        assert np.array_equal(alone[0], m[0])
    ref = oracle.solve(probs[0])
    assert np.abs(mixed[0][0] - ref.x).max() <= TOL32


def test_alone_equals_in_mix():
    """Each request's mesh is bitwise the same alone and in a batch."""
    rng = np.random.default_rng(11)
    probs = W.config4(seed=3, count=12, max_steps=120, size_range=(17, 90))
    probs += [W.small_case(3, 15, parts=(2, 1, 2), overlap=4, steps=50, precision=p)
              for p in ("fp32", "fp64")]
    probs.append(W.config1().replace(max_steps=150))
    mixed = pma.solve_many(probs)
    for k in rng.choice(len(probs), size=6, replace=False):
        alone = pma.solve(probs[k], want_psi=False)
        assert np.array_equal(alone[0], mixed[k][0])
        assert alone[2].steps == mixed[k][2].steps


# ------------------------------------------------------------------ full sizes

@pytest.mark.parametrize("mon", ["ring", "sine"])
def test_config2_full_size(mon):
    """257^2 in 4x4 subdomains (overlap 8), all 16 in one launch: FP64 within
    1e-11 and FP32 within 1e-5 of the oracle after the same 300 steps."""
    p64 = W.config2(mon, "fp64", max_steps=300)
    ref = oracle.solve(p64)
    _check(p64, ref)
    _check(p64.replace(precision="fp32"), ref)


def test_uneven_batch_full_size_sampled():
    """The uneven batch at full size (512 requests, 4,648 subdomains) in one
    context with the bench's launch configuration, capped at 30 steps; the
    largest request and a seeded sample checked one by one against the
    oracle (FP32 sweep against FP64)."""
    probs = [p.replace(max_steps=30) for p in W.config4()]
    res = pma.solve_many(probs, window_steps=128)
    sizes = [p.n[0] * p.n[1] for p in probs]
    rng = np.random.default_rng(14602)
    picks = {int(np.argmax(sizes))} | {int(k) for k in rng.choice(len(probs), 5, replace=False)}
    for k in sorted(picks):
        ref = oracle.solve(probs[k].replace(precision="fp64"))
        x, _, info = res[k]
        assert info.steps == ref.steps, (k, info.steps, ref.steps)
        assert pma.STATUS_NAMES[info.status] == ref.status
        assert np.abs(x - ref.x).max() / _size(probs[k]) <= TOL32, k


@pytest.mark.parametrize("dim,n,parts,o,steps", [(2, (4097, 4097, 1), (2, 2, 1), 8, 4),
                                                 (3, (257, 257, 257), (2, 2, 2), 6, 3)])
def test_large_grids(dim, n, parts, o, steps):
    """Large single requests: 2D subdomains of about 2050 columns (strips of
    several bands across, staged by cp.async), large pitches and plane
    strides; FP64 within 1e-11 and FP32 within 1e-5 of the oracle."""
    p64 = W.Problem(dim=dim, n=n, monitor=W.ring_monitor(dim) if dim == 2 else W.shell_monitor(),
                    parts=parts, overlap=o, dt=W.dt_for(n, dim, cfl=0.1 if dim == 2 else 0.05),
                    tol=0.0, max_steps=steps, precision="fp64")
    ref = oracle.solve(p64)
    _check(p64, ref, psi=False)
    _check(p64.replace(precision="fp32"), ref, psi=False)


def test_config3_full_size_fp32_vs_oracle():
    """129^3 in 2x2x2 subdomains (overlap 6), FP32 sweep vs the FP64 oracle."""
    prob = W.config3("fp32", max_steps=25)
    _check(prob, psi=False)
