"""ctypes wrapper of the C oracle (``pma_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Problems are read by
attribute (dim, n, lo, hi, monitor, parts, overlap, alternating, dt, tol,
max_steps, stop_norm, stop_rule, check_every, rhs, normalize, lag_theta,
exchange_every), so
this module imports nothing from the product package.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pma_oracle.c")
_HDR = os.path.join(_HERE, "pma_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OR_MAX_TERMS = 4

_TERM = {"bump": 0, "ring": 1, "sine": 2, "bump1": 3}
_KIND = {"sum": 0, "product": 1, "arclen_burgers": 2, "arclen_spiral": 3,
         "arclen_tanh_sphere": 4, "arclen_nine_spheres": 5, "table": 6}
_NORM = {"max_ut": 0, "l2_increment": 1}
_RULE = {"all": 0, "any": 1}
_RHS = {"log": 0, "root": 1}
_NRM = {"global_theta": 0, "none": 1}
STATUS = {0: "ok", 1: "not_converged", -1: "invalid", -2: "nomem", -3: "tangled"}


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_long * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3)]


class _Term(C.Structure):
    _fields_ = [("type", C.c_int), ("axis", C.c_int), ("along", C.c_int),
                ("amp", C.c_double), ("width", C.c_double), ("r2", C.c_double),
                ("a", C.c_double), ("k", C.c_double), ("c", C.c_double * 3)]


class _Monitor(C.Structure):
    _fields_ = [("kind", C.c_int), ("nterms", C.c_int), ("base", C.c_double),
                ("p0", C.c_double), ("term", _Term * OR_MAX_TERMS),
                ("table", C.POINTER(C.c_double)), ("tn", C.c_int * 3),
                ("tlo", C.c_double * 3), ("thi", C.c_double * 3)]


class _Decomp(C.Structure):
    _fields_ = [("parts", C.c_int * 3), ("overlap", C.c_int), ("alternating", C.c_int),
                ("exchange_every", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("tol", C.c_double), ("max_steps", C.c_long),
                ("stop_norm", C.c_int), ("stop_rule", C.c_int), ("check_every", C.c_int),
                ("rhs", C.c_int), ("normalize", C.c_int), ("lag_theta", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("steps", C.c_long), ("residual", C.c_double), ("theta", C.c_double),
                ("min_det", C.c_double), ("status", C.c_int)]


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, FP64, no FMA contraction)."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + ".%d.tmp" % os.getpid()
            cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    P = C.POINTER
    lib.or_solve.argtypes = [P(_Grid), P(_Monitor), P(_Decomp), P(_Params),
                             P(C.c_double), P(C.c_double), P(C.c_double),
                             P(C.c_double), P(_Info)]
    lib.or_solve.restype = C.c_int
    lib.or_solve_det.argtypes = [P(_Grid), P(_Monitor), P(_Decomp), P(_Params),
                                 P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                                 P(C.c_double), P(_Info)]
    lib.or_solve_det.restype = C.c_int
    lib.or_monitor_eval.argtypes = [P(_Monitor), C.c_int, P(C.c_double), C.c_long,
                                    P(C.c_double)]
    lib.or_monitor_eval.restype = C.c_int
    lib.or_operator.argtypes = [P(_Grid), P(_Monitor), P(C.c_double), P(C.c_double),
                                P(C.c_double), P(C.c_double), P(C.c_double)]
    lib.or_operator.restype = C.c_int
    lib.or_extents.argtypes = [C.c_long, C.c_int, C.c_int, P(C.c_long), P(C.c_long),
                               P(C.c_long), P(C.c_long)]
    lib.or_extents.restype = C.c_int
    lib.or_quality.argtypes = [P(_Grid), P(_Monitor), P(C.c_double), P(C.c_double)]
    lib.or_quality.restype = C.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(C.CDLL(_LIB))
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every call through another build of the oracle
    source (used by the tests that plant mistakes in a copy of it)."""
    global _lib
    saved = _load()
    _lib = _bind(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _grid(prob) -> _Grid:
    g = _Grid()
    g.dim = prob.dim
    for a in range(3):
        g.n[a] = int(prob.n[a]) if a < prob.dim else 1
        g.lo[a] = float(prob.lo[a])
        g.hi[a] = float(prob.hi[a])
    return g


def _monitor(mon) -> _Monitor:
    m = _Monitor()
    m.kind = _KIND[mon.kind]
    m.nterms = len(mon.terms)
    if m.nterms > OR_MAX_TERMS:
        raise ValueError("at most %d monitor terms" % OR_MAX_TERMS)
    m.base = float(mon.base)
    m.p0 = float(mon.p0)
    for i, t in enumerate(mon.terms):
        T = m.term[i]
        T.type = _TERM[t.type]
        T.axis, T.along = int(t.axis), int(t.along)
        T.amp, T.width, T.r2 = float(t.amp), float(t.width), float(t.r2)
        T.a, T.k = float(t.a), float(t.k)
        for a in range(3):
            T.c[a] = float(t.c[a])
    if mon.kind == "table":
        tab = np.ascontiguousarray(mon.table, dtype=np.float64)
        shape = tab.shape[::-1]  # (tn_x, tn_y[, tn_z])
        for a in range(3):
            m.tn[a] = int(shape[a]) if a < len(shape) else 1
            m.tlo[a] = float(mon.tlo[a])
            m.thi[a] = float(mon.thi[a])
        m.table = tab.ctypes.data_as(C.POINTER(C.c_double))
        m._keep = tab  # the struct holds a raw pointer into this array
    return m


@dataclass
class OracleResult:
    x: np.ndarray          # (dim, N...) mesh, component-major
    psi: np.ndarray        # combined Psi on the global grid
    res: np.ndarray        # residual per step taken
    steps: int
    residual: float
    theta: float
    min_det: float
    status: str
    det: Optional[np.ndarray] = None   # owner-stencil det D_h^2 Psi (want_det)


def _shape(prob):
    return tuple(int(prob.n[a]) for a in reversed(range(prob.dim)))


def solve(prob, psi0: Optional[np.ndarray] = None, want_det: bool = False) -> OracleResult:
    """Run the oracle on a problem (attributes as in the input module);
    want_det also returns det D_h^2 Psi of each global node's owner stencil."""
    lib = _load()
    g = _grid(prob)
    m = _monitor(prob.monitor)
    d = _Decomp()
    for a in range(3):
        d.parts[a] = int(prob.parts[a]) if a < prob.dim else 1
    d.overlap = int(prob.overlap)
    d.alternating = int(prob.alternating)
    d.exchange_every = int(getattr(prob, "exchange_every", 1))
    p = _Params()
    p.dt, p.tol, p.max_steps = float(prob.dt), float(prob.tol), int(prob.max_steps)
    p.stop_norm, p.stop_rule = _NORM[prob.stop_norm], _RULE[prob.stop_rule]
    p.check_every, p.rhs = int(prob.check_every), _RHS[prob.rhs]
    p.normalize, p.lag_theta = _NRM[prob.normalize], int(prob.lag_theta)
    shape = _shape(prob)
    N = int(np.prod(shape))
    x = np.zeros((prob.dim,) + shape, dtype=np.float64)
    psi = np.zeros(shape, dtype=np.float64)
    hist = np.zeros(max(1, int(prob.max_steps)), dtype=np.float64)
    info = _Info()
    p0 = None
    if psi0 is not None:
        p0 = np.ascontiguousarray(psi0, dtype=np.float64).reshape(N)
    det = np.zeros(shape, dtype=np.float64) if want_det else None
    rc = lib.or_solve_det(C.byref(g), C.byref(m), C.byref(d), C.byref(p), _dptr(p0),
                          _dptr(x), _dptr(psi), _dptr(det), _dptr(hist), C.byref(info))
    if rc in (-1, -2):
        raise ValueError("oracle rejected the problem (status %d)" % rc)
    return OracleResult(x=x, psi=psi, res=hist[: info.steps].copy(), steps=int(info.steps),
                        residual=float(info.residual), theta=float(info.theta),
                        min_det=float(info.min_det), status=STATUS[int(info.status)],
                        det=det)


def operator(prob, v: np.ndarray):
    """Single-domain operator on the global grid: (x, det, rho, G)."""
    lib = _load()
    g = _grid(prob)
    m = _monitor(prob.monitor)
    shape = _shape(prob)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(shape)
    x = np.zeros((prob.dim,) + shape)
    det = np.zeros(shape)
    rho = np.zeros(shape)
    G = np.zeros(shape)
    rc = lib.or_operator(C.byref(g), C.byref(m), _dptr(v), _dptr(x), _dptr(det),
                         _dptr(rho), _dptr(G))
    if rc != 0:
        raise ValueError("oracle operator failed (%d)" % rc)
    return x, det, rho, G


def monitor_eval(mon, dim: int, pts: np.ndarray) -> np.ndarray:
    lib = _load()
    m = _monitor(mon)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, dim)
    out = np.zeros(pts.shape[0])
    rc = lib.or_monitor_eval(C.byref(m), dim, _dptr(pts), pts.shape[0], _dptr(out))
    if rc != 0:
        raise ValueError("monitor eval failed")
    return out


def extents(n: int, parts: int, overlap: int):
    lib = _load()
    arrs = [(C.c_long * parts)() for _ in range(4)]
    rc = lib.or_extents(n, parts, overlap, *arrs)
    if rc != 0:
        raise ValueError("invalid decomposition")
    return tuple(np.array(list(a), dtype=np.int64) for a in arrs)


def quality(prob, psi: np.ndarray) -> dict:
    lib = _load()
    g = _grid(prob)
    m = _monitor(prob.monitor)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    out = np.zeros(5)
    rc = lib.or_quality(C.byref(g), C.byref(m), _dptr(psi), _dptr(out))
    if rc != 0:
        raise ValueError("quality failed")
    return {"E2": out[0], "Emax": out[1], "min_det": out[2], "min_cell": out[3],
            "theta": out[4]}


def _solve_job(args):
    prob, psi0 = args
    return solve(prob, psi0)


def solve_parallel(probs, workers: Optional[int] = None, psi0s=None):
    """Run the oracle on several problems at once, one spawned process per
    problem (at most `workers`, default the host's cores up to 16); returns
    the results in order.  Spawned (not forked) workers, so it is safe in a
    process that already uses a GPU."""
    import multiprocessing as mp
    build()
    probs = list(probs)
    if psi0s is None:
        psi0s = [None] * len(probs)
    n = max(1, min(len(probs), workers or min(os.cpu_count() or 1, 16)))
    if n == 1:
        return [solve(p, q) for p, q in zip(probs, psi0s)]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_solve_job, list(zip(probs, psi0s)), chunksize=1)

