"""Seeded synthetic mesh-generation requests.

This module only draws problem descriptions: grids, monitor parameters,
decompositions, time steps and stopping rules.  It holds none of the method's
arithmetic, so both the CUDA library binding and the FP64 test oracle consume
the same inputs from here.

The shapes follow the paper's experiments (Sect. 4): 2D problems on the unit
square from 33^2 up to 1025^2 and 3D problems on cubes, split into 4 or 8
overlapping subdomains (Sects. 4.1-4.3).  The paper's own monitors are the
arc-length densities of analytic test functions (Eq. monitfn with Eqs.
test_fn1, test_fn2, test_fn3d1, test_fn3d2); the synthetic workloads use
Gaussian ring / band / bump densities of the same sharpness instead, and the
paper's functions are available as monitor kinds.

Everything random comes from ``numpy.random.default_rng(seed)``; the master
seed is 14602.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

MASTER_SEED = 14602

# term / monitor / option vocabulary (names, not arithmetic)
TERM_TYPES = ("bump", "ring", "sine", "bump1")
MONITOR_KINDS = ("sum", "product", "arclen_burgers", "arclen_spiral",
                 "arclen_tanh_sphere", "arclen_nine_spheres")
STOP_NORMS = ("max_ut", "l2_increment")
STOP_RULES = ("all", "any")
RHS_FORMS = ("log", "root")
NORMALIZE = ("global_theta", "none")
PRECISIONS = ("fp32", "fp64")


@dataclass
class Term:
    """One term of a monitor density (see the monitor kinds)."""
    type: str = "bump"
    amp: float = 1.0
    width: float = 1.0
    r2: float = 0.0
    c: Tuple[float, float, float] = (0.5, 0.5, 0.5)
    a: float = 0.0
    k: float = 0.0
    axis: int = 0
    along: int = 0


@dataclass
class Monitor:
    kind: str = "sum"
    base: float = 1.0
    terms: List[Term] = field(default_factory=list)
    p0: float = 0.0
    # kind "table": density values on a uniform grid over [tlo, thi], array
    # shaped (n_y, n_x) or (n_z, n_y, n_x)
    table: Optional[np.ndarray] = field(default=None, compare=False, repr=False)
    tlo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    thi: Tuple[float, float, float] = (1.0, 1.0, 1.0)


@dataclass
class Problem:
    """One mesh-generation request: the paper's problem statement
    (domain and grid, monitor, subdomains and overlap, time step and
    stopping rule; Sects. 2-3)."""
    dim: int
    n: Tuple[int, int, int]
    lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    hi: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    monitor: Monitor = field(default_factory=Monitor)
    parts: Tuple[int, int, int] = (1, 1, 1)
    overlap: int = 0
    alternating: int = 0
    exchange_every: int = 1
    dt: float = 1e-4
    tol: float = 1e-6
    max_steps: int = 2000
    stop_norm: str = "max_ut"
    stop_rule: str = "all"
    check_every: int = 1
    rhs: str = "log"
    normalize: str = "global_theta"
    lag_theta: int = 0
    precision: str = "fp64"

    @property
    def nodes(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _h2(n: Sequence[int], lo, hi, dim: int) -> float:
    """Smallest squared grid spacing (a parameter of the dt choice only)."""
    return min(((hi[a] - lo[a]) / (n[a] - 1)) ** 2 for a in range(dim))


def dt_for(n, dim: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), cfl: float = 0.1) -> float:
    """Pseudo-time step dt = cfl * min h^2 (Sect. 4.4 uses 0.015..0.12 h^2)."""
    return cfl * _h2(n, lo, hi, dim)


# --------------------------------------------------------------------------
# monitors of the synthetic configurations
# --------------------------------------------------------------------------

def ring_monitor(dim: int = 2, amp: float = 10.0, width: float = 50.0,
                 r2: float = 0.0625, centre=(0.5, 0.5, 0.5)) -> Monitor:
    return Monitor("sum", 1.0, [Term("ring", amp, width, r2, tuple(centre))])


def sine_monitor(amp: float = 5.0, width: float = 100.0) -> Monitor:
    """rho = 1 + 5 exp(-100 (x2 - 0.5 - 0.25 sin(2 pi x1))^2)."""
    return Monitor("sum", 1.0, [Term("sine", amp, width, 0.0, (0.5, 0.5, 0.5),
                                     a=0.25, k=1.0, axis=1, along=0)])


def shell_monitor() -> Monitor:
    """rho = 1 + 20 exp(-80 (|x - c|^2 - 0.09)^2), c = (0.5, 0.5, 0.5)."""
    return ring_monitor(3, 20.0, 80.0, 0.09, (0.5, 0.5, 0.5))


def uniform_monitor(value: float = 1.0) -> Monitor:
    return Monitor("sum", value, [])


def product_monitor(factors: Sequence[Tuple[float, float, float]]) -> Monitor:
    """Separable rho = prod_a (1 + amp_a exp(-width_a (x_a - c_a)^2))."""
    terms = []
    for a, (amp, width, c) in enumerate(factors):
        cc = [0.5, 0.5, 0.5]
        cc[a] = c
        terms.append(Term("bump1", amp, width, 0.0, tuple(cc), axis=a))
    return Monitor("product", 1.0, terms)


def random_bumps(rng: np.random.Generator, dim: int, nterms: Optional[int] = None) -> Monitor:
    """1-4 Gaussian bumps/rings, amplitudes U[1,50], widths U[20,200],
    centres U[0.2,0.8]^d; ring radii r^2 ~ U[0.01, 0.09]."""
    if nterms is None:
        nterms = int(rng.integers(1, 5))
    terms = []
    for _ in range(nterms):
        amp = float(rng.uniform(1.0, 50.0))
        width = float(rng.uniform(20.0, 200.0))
        c = [0.5, 0.5, 0.5]
        for a in range(dim):
            c[a] = float(rng.uniform(0.2, 0.8))
        if rng.uniform() < 0.5:
            terms.append(Term("bump", amp, width, 0.0, tuple(c)))
        else:
            terms.append(Term("ring", amp, width, float(rng.uniform(0.01, 0.09)), tuple(c)))
    return Monitor("sum", 1.0, terms)


# --------------------------------------------------------------------------
# the five configurations
# --------------------------------------------------------------------------

def config1(precision: str = "fp64") -> Problem:
    """2D single domain, 33x33, ring monitor, dt = 1e-4, max|u_t| < 1e-6 or
    2000 steps."""
    return Problem(dim=2, n=(33, 33, 1), monitor=ring_monitor(), dt=1e-4, tol=1e-6,
                   max_steps=2000, precision=precision)


def config2(monitor: str = "ring", precision: str = "fp32", max_steps: int = 2000,
            cfl: float = 0.1) -> Problem:
    """2D 257x257 in 4x4 overlapping subdomains, overlap 8."""
    mon = ring_monitor() if monitor == "ring" else sine_monitor()
    n = (257, 257, 1)
    return Problem(dim=2, n=n, monitor=mon, parts=(4, 4, 1), overlap=8,
                   dt=dt_for(n, 2, cfl=cfl), tol=1e-6, max_steps=max_steps,
                   precision=precision)


def config3(precision: str = "fp32", max_steps: int = 2000, cfl: float = 0.05) -> Problem:
    """3D 129^3 in 2x2x2 subdomains, overlap 6, spherical shell monitor."""
    n = (129, 129, 129)
    return Problem(dim=3, n=n, monitor=shell_monitor(), parts=(2, 2, 2), overlap=6,
                   dt=dt_for(n, 3, cfl=cfl), tol=1e-6, max_steps=max_steps,
                   precision=precision)


def _parts_for(rng: np.random.Generator, n: int, overlap: int, max_parts: int) -> int:
    """Largest admissible part count drawn uniformly, each core keeping at
    least max(overlap + 2, 8) nodes."""
    core_min = max(overlap + 2, 8)
    pmax = max(1, min(max_parts, n // core_min))
    return int(rng.integers(1, pmax + 1))


def config4(seed: int = MASTER_SEED, count: int = 512, precision: str = "fp32",
            max_steps: int = 2000, cfl: float = 0.1,
            size_range: Tuple[int, int] = (17, 513)) -> List[Problem]:
    """512 independent 2D problems: per-side sizes log-uniform in [17, 513],
    1-16 subdomains (px * py <= 16), overlap 4-8, random bump/ring sums."""
    rng = np.random.default_rng(seed)
    out = []
    lo_s, hi_s = math.log(size_range[0]), math.log(size_range[1])
    for _ in range(count):
        nx = int(round(math.exp(rng.uniform(lo_s, hi_s))))
        ny = int(round(math.exp(rng.uniform(lo_s, hi_s))))
        o = int(rng.integers(4, 9))
        px = _parts_for(rng, nx, o, 16)
        py = _parts_for(rng, ny, o, max(1, 16 // px))
        if px * py == 1:
            o = 0
        n = (nx, ny, 1)
        out.append(Problem(dim=2, n=n, monitor=random_bumps(rng, 2), parts=(px, py, 1),
                           overlap=o, dt=dt_for(n, 2, cfl=cfl), tol=1e-6,
                           max_steps=max_steps, precision=precision))
    return out


def config5_stream(seed: int = MASTER_SEED, count: int = 256, rate_hz: float = 100.0,
                   precision: str = "fp32", max_steps: int = 2000,
                   size2d: Tuple[int, int] = (33, 1025),
                   size3d: Tuple[int, int] = (17, 193),
                   frac3d: float = 0.2) -> List[Tuple[float, Problem]]:
    """Poisson arrivals of mixed 2D / 3D requests, 1-27 subdomains, random
    bump monitors; returns (arrival time in s, problem) pairs."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        if rng.uniform() < frac3d:
            dim = 3
            lo_s, hi_s = math.log(size3d[0]), math.log(size3d[1])
            side = int(round(math.exp(rng.uniform(lo_s, hi_s))))
            n = (side, side, side)
            o = int(rng.integers(4, 9))
            p = _parts_for(rng, side, o, 3)
            parts = (p, p, p)
            cfl = 0.05
        else:
            dim = 2
            lo_s, hi_s = math.log(size2d[0]), math.log(size2d[1])
            side = int(round(math.exp(rng.uniform(lo_s, hi_s))))
            n = (side, side, 1)
            o = int(rng.integers(4, 9))
            px = _parts_for(rng, side, o, 5)
            py = _parts_for(rng, side, o, max(1, 25 // px))
            parts = (px, py, 1)
            cfl = 0.1
        if parts[0] * parts[1] * parts[2] == 1:
            o = 0
        out.append((t, Problem(dim=dim, n=n, monitor=random_bumps(rng, dim), parts=parts,
                               overlap=o, dt=dt_for(n, dim, cfl=cfl), tol=1e-6,
                               max_steps=max_steps, precision=precision)))
    return out


def small_case(dim: int = 2, n: int = 21, parts=(1, 1, 1), overlap: int = 0,
               monitor: Optional[Monitor] = None, steps: int = 50, cfl: float = 0.1,
               precision: str = "fp64") -> Problem:
    """A small problem the oracle finishes in well under a second."""
    nn = (n, n if dim > 1 else 1, n if dim > 2 else 1)
    if monitor is None:
        monitor = ring_monitor(dim) if dim > 1 else Monitor(
            "sum", 1.0, [Term("bump", 10.0, 50.0, 0.0, (0.5, 0.5, 0.5))])
    return Problem(dim=dim, n=nn, monitor=monitor, parts=tuple(parts), overlap=overlap,
                   dt=dt_for(nn, dim, cfl=cfl), tol=0.0, max_steps=steps,
                   precision=precision)
