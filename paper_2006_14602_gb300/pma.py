"""Thin ctypes binding of the C ABI in ``include/pma.h``.

Every ``pma_*`` function of the header is exposed under the same name with
argument marshalling only; all computation happens in ``libpma.so`` (the
sm_103a kernels and their host runtime).  There is no Python or CPU fallback:
if the library has not been built, importing its functions raises.

``Context`` and ``solve`` are conveniences that convert the problem
descriptions of :mod:`paper_2006_14602_gb300.workloads` into the C structs.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Iterable, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpma.so")

PMA_MAX_TERMS = 4
PMA_MAX_PARTS = 32

# status codes
PMA_OK = 0
PMA_NOT_CONVERGED = 1
PMA_PENDING = 2
PMA_ERR_INVALID = -1
PMA_ERR_NOMEM = -2
PMA_ERR_TANGLED = -3
PMA_ERR_TIMEOUT = -4
PMA_ERR_CUDA = -5
PMA_ERR_BUSY = -6
PMA_ERR_NOT_FOUND = -7
STATUS_NAMES = {0: "ok", 1: "not_converged", 2: "pending", -1: "invalid", -2: "nomem",
                -3: "tangled", -4: "timeout", -5: "cuda", -6: "busy", -7: "not_found"}

# options
PMA_OPT_WINDOW_STEPS = 1
PMA_OPT_USE_GRAPHS = 2
PMA_OPT_LAUNCH_MODE = 3
PMA_OPT_TILE_2D = 4
PMA_OPT_TILE_3D = 5
PMA_OPT_MAX_ACTIVE = 6
PMA_OPT_RESIDENT = 7
PMA_OPT_TIME_SWEEPS = 8
PMA_OPT_RESIDENT_STEPS = 9
PMA_OPT_TEST_STALL = 10
PMA_OPT_GROUPS = 11
PMA_LAUNCH_BATCHED = 0
PMA_LAUNCH_PER_SUBDOMAIN = 1

_TERM = {"bump": 0, "ring": 1, "sine": 2, "bump1": 3}
_KIND = {"sum": 0, "product": 1, "arclen_burgers": 2, "arclen_spiral": 3,
         "arclen_tanh_sphere": 4, "arclen_nine_spheres": 5, "table": 6}
_NORM = {"max_ut": 0, "l2_increment": 1}
_RULE = {"all": 0, "any": 1}
_RHS = {"log": 0, "root": 1}
_NRM = {"global_theta": 0, "none": 1}
_PREC = {"fp32": 0, "fp64": 1}


class pma_grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3)]


class pma_term(C.Structure):
    _fields_ = [("type", C.c_int32), ("axis", C.c_int32), ("along", C.c_int32),
                ("reserved", C.c_int32), ("amp", C.c_double), ("width", C.c_double),
                ("r2", C.c_double), ("a", C.c_double), ("k", C.c_double),
                ("c", C.c_double * 3)]


class pma_monitor(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nterms", C.c_int32), ("base", C.c_double),
                ("p0", C.c_double), ("term", pma_term * PMA_MAX_TERMS),
                ("table", C.POINTER(C.c_double)), ("tn", C.c_int32 * 3),
                ("reserved", C.c_int32), ("tlo", C.c_double * 3), ("thi", C.c_double * 3)]


class pma_decomp(C.Structure):
    _fields_ = [("parts", C.c_int32 * 3), ("overlap", C.c_int32),
                ("transmission", C.c_int32), ("exchange_every", C.c_int32)]


class pma_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("tol", C.c_double), ("max_steps", C.c_int64),
                ("stop_norm", C.c_int32), ("stop_rule", C.c_int32),
                ("check_every", C.c_int32), ("rhs", C.c_int32), ("normalize", C.c_int32),
                ("precision", C.c_int32)]


class pma_info(C.Structure):
    _fields_ = [("steps", C.c_int64), ("residual", C.c_double), ("theta", C.c_double),
                ("min_det", C.c_double), ("shift", C.c_double), ("status", C.c_int32),
                ("reserved", C.c_int32), ("latency_us", C.c_double)]


class pma_stats(C.Structure):
    _fields_ = [("windows", C.c_int64), ("sweep_launches", C.c_int64),
                ("other_launches", C.c_int64), ("node_updates", C.c_int64),
                ("sweep_bytes", C.c_double), ("window_ms", C.c_double),
                ("h2d_bytes", C.c_double), ("d2h_bytes", C.c_double),
                ("res_launches", C.c_int64), ("res_node_updates", C.c_int64),
                ("sweep_kernel_ms", C.c_double), ("sweep_kernel_launches", C.c_int64),
                ("admit_ms", C.c_double), ("rebuild_ms", C.c_double),
                ("combine_ms", C.c_double), ("sweep_steps", C.c_int64)]


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes)
_P = C.POINTER
_SIGS = {
    "pma_status_str": (C.c_char_p, [C.c_int32]),
    "pma_last_error": (C.c_char_p, []),
    "pma_abi_version": (C.c_int32, []),
    "pma_selftest_tables": (C.c_int32, []),
    "pma_create": (C.c_int, [_P(C.c_void_p), C.c_int, C.c_size_t, C.c_void_p]),
    "pma_destroy": (C.c_int, [C.c_void_p]),
    "pma_set_option": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "pma_get_option": (C.c_int, [C.c_void_p, C.c_int32, _P(C.c_int64)]),
    "pma_submit": (C.c_int, [C.c_void_p, _P(pma_grid), _P(pma_monitor), _P(pma_decomp),
                             _P(pma_params), _P(C.c_double), _P(C.c_uint64)]),
    "pma_run": (C.c_int, [C.c_void_p, C.c_int64, _P(C.c_int32)]),
    "pma_serve_start": (C.c_int, [C.c_void_p]),
    "pma_serve_stop": (C.c_int, [C.c_void_p]),
    "pma_admit": (C.c_int, [C.c_void_p]),
    "pma_get_mesh_device_batch": (C.c_int, [C.c_void_p, C.c_int32, _P(C.c_uint64),
                                            _P(C.c_void_p), C.c_int32]),
    "pma_get_mesh_batch": (C.c_int, [C.c_void_p, C.c_int32, _P(C.c_uint64), _P(C.c_double),
                                     _P(pma_info)]),
    "pma_get_stats": (C.c_int, [C.c_void_p, _P(pma_stats), C.c_int32]),
    "pma_poll": (C.c_int, [C.c_void_p, C.c_uint64, _P(C.c_int32)]),
    "pma_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int64]),
    "pma_get_mesh": (C.c_int, [C.c_void_p, C.c_uint64, _P(C.c_double), _P(C.c_double),
                               _P(pma_info)]),
    "pma_get_mesh_device": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int32,
                                      C.c_void_p, _P(pma_info)]),
    "pma_check_mesh": (C.c_int, [C.c_void_p, C.c_uint64, _P(C.c_double)]),
    "pma_get_info": (C.c_int, [C.c_void_p, C.c_uint64, _P(pma_info)]),
    "pma_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "pma_counts": (C.c_int, [C.c_void_p, _P(C.c_int32), _P(C.c_int32), _P(C.c_int32)]),
    "pma_solve": (C.c_int, [C.c_int, _P(pma_grid), _P(pma_monitor), _P(pma_decomp),
                            _P(pma_params), _P(C.c_double), _P(C.c_double), _P(C.c_double),
                            _P(pma_info)]),
    "pma_solve_static": (C.c_int, [_P(pma_grid), _P(pma_monitor), _P(pma_decomp),
                                   _P(pma_params), C.c_void_p, C.c_void_p, _P(pma_info),
                                   C.c_void_p]),
}


def exported_symbols() -> List[str]:
    return sorted(_SIGS)


def load(path: Optional[str] = None):
    """Load libpma.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError("libpma.so is not built (%s); run "
                                   "paper_2006_14602_gb300.build.build()" % p)
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _call(name, *args):
    return getattr(load(), name)(*args)


# ---- same-name wrappers (marshalling only) --------------------------------

def pma_status_str(s: int) -> str:
    return _call("pma_status_str", s).decode()


def pma_last_error() -> str:
    return _call("pma_last_error").decode()


def pma_abi_version() -> int:
    return _call("pma_abi_version")


def pma_selftest_tables() -> int:
    """Host-only consistency checks of the device tables (no GPU used);
    returns the number of failed checks."""
    return _call("pma_selftest_tables")


def pma_create(device: int = 0, mem_budget_bytes: int = 0, cuda_stream: int = 0):
    h = C.c_void_p()
    st = _call("pma_create", C.byref(h), device, mem_budget_bytes, C.c_void_p(cuda_stream or None))
    return st, h


def pma_destroy(ctx) -> int:
    return _call("pma_destroy", ctx)


def pma_set_option(ctx, opt: int, value: int) -> int:
    return _call("pma_set_option", ctx, opt, value)


def pma_get_option(ctx, opt: int):
    v = C.c_int64()
    st = _call("pma_get_option", ctx, opt, C.byref(v))
    return st, v.value


def pma_submit(ctx, grid, monitor, decomp, params, psi0: Optional[np.ndarray] = None):
    rid = C.c_uint64()
    p0 = None
    if psi0 is not None:
        psi0 = np.ascontiguousarray(psi0, dtype=np.float64)
        p0 = psi0.ctypes.data_as(_P(C.c_double))
    st = _call("pma_submit", ctx, C.byref(grid), C.byref(monitor),
               C.byref(decomp) if decomp is not None else None, C.byref(params), p0,
               C.byref(rid))
    return st, rid.value


def pma_run(ctx, max_windows: int = 0):
    n = C.c_int32()
    st = _call("pma_run", ctx, max_windows, C.byref(n))
    return st, n.value


def pma_serve_start(ctx) -> int:
    return _call("pma_serve_start", ctx)


def pma_serve_stop(ctx) -> int:
    return _call("pma_serve_stop", ctx)


def pma_admit(ctx) -> int:
    return _call("pma_admit", ctx)


def pma_get_mesh_device_batch(ctx, ids: Sequence[int], x_dev_ptrs: Sequence[int],
                              out_fp64: int = 1) -> int:
    n = len(ids)
    a = (C.c_uint64 * max(n, 1))(*ids)
    b = (C.c_void_p * max(n, 1))(*[C.c_void_p(p) for p in x_dev_ptrs])
    return _call("pma_get_mesh_device_batch", ctx, n, a, b, out_fp64)


def pma_get_mesh_batch(ctx, ids: Sequence[int], x_out_ptr: int, infos=None) -> int:
    """Meshes of finished requests packed back to back into one host buffer
    at address x_out_ptr (doubles); infos: optional ctypes array of pma_info
    with len(ids) entries."""
    n = len(ids)
    a = (C.c_uint64 * max(n, 1))(*ids)
    return _call("pma_get_mesh_batch", ctx, n, a, C.cast(C.c_void_p(x_out_ptr), _P(C.c_double)),
                 infos)


def pma_get_stats(ctx, reset: int = 0):
    s = pma_stats()
    st = _call("pma_get_stats", ctx, C.byref(s), reset)
    return st, s


def pma_poll(ctx, rid: int):
    d = C.c_int32()
    st = _call("pma_poll", ctx, rid, C.byref(d))
    return st, d.value


def pma_wait(ctx, rid: int, timeout_us: int = -1) -> int:
    return _call("pma_wait", ctx, rid, timeout_us)


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.flags["WRITEABLE"]
    return a.ctypes.data_as(_P(C.c_double))


def pma_get_mesh(ctx, rid: int, x_out: np.ndarray, psi_out: Optional[np.ndarray] = None):
    info = pma_info()
    st = _call("pma_get_mesh", ctx, rid, _dp(x_out), _dp(psi_out), C.byref(info))
    return st, info


def pma_get_mesh_device(ctx, rid: int, x_dev_ptr: int, out_fp64: int = 1,
                        psi_dev_ptr: int = 0):
    info = pma_info()
    st = _call("pma_get_mesh_device", ctx, rid, C.c_void_p(x_dev_ptr), out_fp64,
               C.c_void_p(psi_dev_ptr or None), C.byref(info))
    return st, info


def pma_check_mesh(ctx, rid: int):
    out = (C.c_double * 4)()
    st = _call("pma_check_mesh", ctx, rid, out)
    return st, list(out)


def pma_get_info(ctx, rid: int):
    info = pma_info()
    st = _call("pma_get_info", ctx, rid, C.byref(info))
    return st, info


def pma_release(ctx, rid: int) -> int:
    return _call("pma_release", ctx, rid)


def pma_counts(ctx):
    q, a, f = C.c_int32(), C.c_int32(), C.c_int32()
    st = _call("pma_counts", ctx, C.byref(q), C.byref(a), C.byref(f))
    return st, (q.value, a.value, f.value)


def pma_solve(device, grid, monitor, decomp, params, psi0, x_out, psi_out=None):
    info = pma_info()
    p0 = None
    if psi0 is not None:
        psi0 = np.ascontiguousarray(psi0, dtype=np.float64)
        p0 = psi0.ctypes.data_as(_P(C.c_double))
    st = _call("pma_solve", device, C.byref(grid), C.byref(monitor),
               C.byref(decomp) if decomp is not None else None, C.byref(params), p0,
               _dp(x_out), _dp(psi_out), C.byref(info))
    return st, info


# ---- struct conversion from the input module's problem descriptions -------

def to_structs(prob):
    """(grid, monitor, decomp, params) C structs of a Problem."""
    g = pma_grid()
    g.dim = prob.dim
    for a in range(3):
        g.n[a] = int(prob.n[a]) if a < prob.dim else 1
        g.lo[a] = float(prob.lo[a])
        g.hi[a] = float(prob.hi[a])
    m = pma_monitor()
    mon = prob.monitor
    m.kind = _KIND[mon.kind]
    m.nterms = len(mon.terms)
    if m.nterms > PMA_MAX_TERMS:
        raise ValueError("at most %d monitor terms" % PMA_MAX_TERMS)
    m.base = float(mon.base)
    m.p0 = float(mon.p0)
    for i, t in enumerate(mon.terms):
        T = m.term[i]
        T.type = _TERM[t.type]
        T.axis, T.along = int(t.axis), int(t.along)
        T.amp, T.width, T.r2, T.a, T.k = (float(t.amp), float(t.width), float(t.r2),
                                          float(t.a), float(t.k))
        for a in range(3):
            T.c[a] = float(t.c[a])
    if mon.kind == "table":
        tab = np.ascontiguousarray(mon.table, dtype=np.float64)
        shape = tab.shape[::-1]  # (n_x, n_y[, n_z])
        for a in range(3):
            m.tn[a] = int(shape[a]) if a < len(shape) else 1
            m.tlo[a] = float(mon.tlo[a])
            m.thi[a] = float(mon.thi[a])
        m.table = tab.ctypes.data_as(C.POINTER(C.c_double))
        m._keep = tab  # copied by the library at submit
    d = pma_decomp()
    for a in range(3):
        d.parts[a] = int(prob.parts[a]) if a < prob.dim else 1
    d.overlap = int(prob.overlap)
    d.transmission = int(prob.alternating)
    d.exchange_every = int(getattr(prob, "exchange_every", 1))
    p = pma_params()
    p.dt, p.tol, p.max_steps = float(prob.dt), float(prob.tol), int(prob.max_steps)
    p.stop_norm, p.stop_rule = _NORM[prob.stop_norm], _RULE[prob.stop_rule]
    p.check_every, p.rhs = int(prob.check_every), _RHS[prob.rhs]
    p.normalize, p.precision = _NRM[prob.normalize], _PREC[prob.precision]
    if prob.rhs == "root" and not int(prob.lag_theta):
        raise ValueError("the device root form uses theta of the previous step "
                         "(lag_theta=1)")
    return g, m, d, p


class PmaError(RuntimeError):
    def __init__(self, call, st):
        super().__init__("%s failed: %s (%s)" % (call, STATUS_NAMES.get(st, st),
                                                 pma_last_error()))
        self.status = st


def _shape(prob):
    return tuple(int(prob.n[a]) for a in reversed(range(prob.dim)))


class Context:
    """Owning wrapper of a pma_ctx."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, cuda_stream: int = 0,
                 **options):
        st, self.h = pma_create(device, mem_budget_bytes, cuda_stream)
        if st != PMA_OK:
            raise PmaError("pma_create", st)
        for k, v in options.items():
            self.set(k, v)

    _OPTS = {"window_steps": PMA_OPT_WINDOW_STEPS, "use_graphs": PMA_OPT_USE_GRAPHS,
             "launch_mode": PMA_OPT_LAUNCH_MODE, "tile_2d": PMA_OPT_TILE_2D,
             "tile_3d": PMA_OPT_TILE_3D, "max_active": PMA_OPT_MAX_ACTIVE,
             "resident": PMA_OPT_RESIDENT, "time_sweeps": PMA_OPT_TIME_SWEEPS,
             "resident_steps": PMA_OPT_RESIDENT_STEPS, "test_stall": PMA_OPT_TEST_STALL,
             "groups": PMA_OPT_GROUPS}

    def set(self, name: str, value: int):
        st = pma_set_option(self.h, self._OPTS[name], int(value))
        if st != PMA_OK:
            raise PmaError("pma_set_option(%s)" % name, st)

    def submit(self, prob, psi0: Optional[np.ndarray] = None) -> int:
        g, m, d, p = to_structs(prob)
        st, rid = pma_submit(self.h, g, m, d, p, psi0)
        if st != PMA_OK:
            raise PmaError("pma_submit", st)
        return rid

    def run(self, max_windows: int = 0) -> int:
        st, n = pma_run(self.h, max_windows)
        if st != PMA_OK:
            raise PmaError("pma_run", st)
        return n

    def mesh(self, prob, rid: int, want_psi: bool = False):
        shape = _shape(prob)
        x = np.empty((prob.dim,) + shape, dtype=np.float64)
        psi = np.empty(shape, dtype=np.float64) if want_psi else None
        st, info = pma_get_mesh(self.h, rid, x, psi)
        if st not in (PMA_OK, PMA_NOT_CONVERGED, PMA_ERR_TANGLED):
            raise PmaError("pma_get_mesh", st)
        return x, psi, info

    def close(self):
        if getattr(self, "h", None):
            pma_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(prob, psi0: Optional[np.ndarray] = None, device: int = 0, want_psi: bool = True,
          **options):
    """Run one problem to completion on the device; returns (x, psi, info)."""
    with Context(device, **options) as ctx:
        rid = ctx.submit(prob, psi0)
        ctx.run()
        return ctx.mesh(prob, rid, want_psi)


def solve_many(probs: Sequence, device: int = 0, want_psi: bool = False, **options):
    """Run several problems in one batched context; list of (x, psi, info)."""
    with Context(device, **options) as ctx:
        ids = [ctx.submit(p) for p in probs]
        ctx.run()
        return [ctx.mesh(p, i, want_psi) for p, i in zip(probs, ids)]


PMA_STATIC_SCRATCH_BYTES = 32 << 20


def pma_solve_static(grid, monitor, decomp, params, psi0_dev_ptr: int, x_dev_ptr: int,
                     cuda_stream: int = 0):
    """Allocation-free solve: device pointers in and out, fixed library scratch."""
    info = pma_info()
    st = _call("pma_solve_static", C.byref(grid), C.byref(monitor),
               C.byref(decomp) if decomp is not None else None, C.byref(params),
               C.c_void_p(psi0_dev_ptr or None), C.c_void_p(x_dev_ptr), C.byref(info),
               C.c_void_p(cuda_stream or None))
    return st, info
