"""ctypes binding of libpf (include/pf.h): argument marshalling only.

Every function keeps the C name and signature; pointers are passed as
integers (device pointers from torch tensors, host pointers from numpy
arrays or pinned torch tensors). Every step of the computation runs in the
CUDA library; there is no Python or CPU fallback, and importing this module
raises if libpf.so has not been built.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpf.so")

PF_OK, PF_ERR_INVALID, PF_ERR_CUDA, PF_ERR_NOT_CONVERGED = 0, 1, 2, 3
PF_ERR_NONFINITE, PF_ERR_UNBOUNDED, PF_ERR_TIMEOUT, PF_ERR_WORKSPACE = 4, 5, 6, 7
STATUS_NAMES = {0: "PF_OK", 1: "PF_ERR_INVALID", 2: "PF_ERR_CUDA", 3: "PF_ERR_NOT_CONVERGED",
                4: "PF_ERR_NONFINITE", 5: "PF_ERR_UNBOUNDED", 6: "PF_ERR_TIMEOUT",
                7: "PF_ERR_WORKSPACE"}
PF_FIELD_PHI, PF_FIELD_U, PF_FIELD_V, PF_FIELD_W, PF_FIELD_P = 0, 1, 2, 3, 4

# Exported symbols declared in include/pf.h (checked by the CPU test suite).
SYMBOLS = ["pf_workspace_size", "pf_init", "pf_step", "pf_project", "pf_diagnostics",
           "pf_get_field", "pf_set_field", "pf_state_bytes", "pf_get_state", "pf_set_state",
           "pf_eval_rhs", "pf_poisson_solve", "pf_sync", "pf_destroy", "pf_last_error",
           "pf_profile_enable", "pf_profile_read", "pf_poisson_solve_static",
           "pf_batch_workspace_size", "pf_batch_init", "pf_batch_step", "pf_batch_step_each",
           "pf_batch_size",
           "pf_batch_context", "pf_batch_destroy", "pf_batch_last_error",
           "pf_adjoint_workspace_size", "pf_step_adjoint", "pf_objective"]


class pf_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double),
        ("model", ctypes.c_int), ("force", ctypes.c_int), ("precision", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("sigma", ctypes.c_double), ("eps", ctypes.c_double),
        ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
        ("mu_in", ctypes.c_double), ("mu_out", ctypes.c_double),
        ("gamma_fixed", ctypes.c_double), ("gamma_min", ctypes.c_double),
        ("dt", ctypes.c_double), ("delta_n", ctypes.c_double),
        ("poisson_rtol", ctypes.c_double), ("poisson_maxit", ctypes.c_int),
        ("R", ctypes.c_double), ("pert_mode", ctypes.c_int), ("pert_amp", ctypes.c_double),
        ("mg_pre", ctypes.c_int), ("mg_post", ctypes.c_int),
        ("bound_tol", ctypes.c_double),
        ("inner_tol", ctypes.c_double),
        ("use_graph", ctypes.c_int),
        ("momentum", ctypes.c_int),
        ("wall_y", ctypes.c_int),
        ("shape", ctypes.c_int),
        ("mg_coarse_cells", ctypes.c_int),
        ("sweep_staging", ctypes.c_int),
        ("stage_kernel", ctypes.c_int),
        ("sweep_tile", ctypes.c_int),
        ("reserved", ctypes.c_int * 1),
    ]


class pf_diag(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("ke", ctypes.c_double), ("se", ctypes.c_double),
        ("umax", ctypes.c_double), ("ca_inf", ctypes.c_double), ("dp_laplace", ctypes.c_double),
        ("phi_min", ctypes.c_double), ("phi_max", ctypes.c_double),
        ("poisson_relres", ctypes.c_double), ("gamma", ctypes.c_double),
        ("poisson_iters", ctypes.c_int), ("poisson_iters_max", ctypes.c_int),
        ("step", ctypes.c_longlong), ("t", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pf_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double)]


class PFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, sz, i32, f64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "pf_workspace_size": (i32, [P(pf_params), P(sz)]),
        "pf_init": (i32, [P(pf_params), vp, sz, vp, vp, P(vp)]),
        "pf_step": (i32, [vp, i32]),
        "pf_project": (i32, [vp]),
        "pf_diagnostics": (i32, [vp, P(pf_diag)]),
        "pf_get_field": (i32, [vp, i32, vp]),
        "pf_set_field": (i32, [vp, i32, vp]),
        "pf_state_bytes": (sz, [vp]),
        "pf_get_state": (i32, [vp, vp]),
        "pf_set_state": (i32, [vp, vp]),
        "pf_eval_rhs": (i32, [vp, f64, vp, vp]),
        "pf_poisson_solve": (i32, [vp, vp, vp, P(i32), P(f64)]),
        "pf_sync": (i32, [vp]),
        "pf_destroy": (None, [vp]),
        "pf_last_error": (ctypes.c_char_p, [vp]),
        "pf_profile_enable": (i32, [vp, i32]),
        "pf_profile_read": (i32, [vp, P(pf_profile_entry), i32, i32]),
        "pf_poisson_solve_static": (i32, [P(pf_params), vp, vp, vp, vp, P(i32), P(f64)]),
        "pf_batch_workspace_size": (i32, [P(pf_params), i32, P(sz)]),
        "pf_batch_init": (i32, [P(pf_params), i32, vp, sz, i32, P(vp)]),
        "pf_batch_step": (i32, [vp, i32]),
        "pf_batch_step_each": (i32, [vp, P(i32)]),
        "pf_batch_size": (i32, [vp]),
        "pf_batch_context": (vp, [vp, i32]),
        "pf_batch_destroy": (None, [vp]),
        "pf_batch_last_error": (ctypes.c_char_p, [vp]),
        "pf_adjoint_workspace_size": (i32, [P(pf_params), P(sz)]),
        "pf_step_adjoint": (i32, [vp, vp, sz, vp, vp, vp]),
        "pf_objective": (i32, [vp, vp, f64, f64, P(f64), vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def _check(status, ctx=None):
    if status != PF_OK:
        msg = LIB.pf_last_error(ctx)
        raise PFError(status, msg.decode() if msg else "")
    return status


def pf_workspace_size(params: pf_params) -> int:
    n = ctypes.c_size_t(0)
    _check(LIB.pf_workspace_size(ctypes.byref(params), ctypes.byref(n)))
    return n.value


def pf_init(params: pf_params, workspace: int, workspace_bytes: int, phi0: int | None,
            stream: int | None):
    ctx = ctypes.c_void_p(0)
    _check(LIB.pf_init(ctypes.byref(params), workspace, workspace_bytes, phi0, stream,
                       ctypes.byref(ctx)))
    return ctx


def pf_step(ctx, nsteps: int):
    return _check(LIB.pf_step(ctx, nsteps), ctx)


def pf_project(ctx):
    return _check(LIB.pf_project(ctx), ctx)


def pf_diagnostics(ctx) -> dict:
    d = pf_diag()
    _check(LIB.pf_diagnostics(ctx, ctypes.byref(d)), ctx)
    return d.as_dict()


def pf_get_field(ctx, field: int, dst: int):
    return _check(LIB.pf_get_field(ctx, field, dst), ctx)


def pf_set_field(ctx, field: int, src: int):
    return _check(LIB.pf_set_field(ctx, field, src), ctx)


def pf_state_bytes(ctx) -> int:
    return LIB.pf_state_bytes(ctx)


def pf_get_state(ctx, dst: int):
    return _check(LIB.pf_get_state(ctx, dst), ctx)


def pf_set_state(ctx, src: int):
    return _check(LIB.pf_set_state(ctx, src), ctx)


def pf_eval_rhs(ctx, gamma: float, kphi: int, ku: int):
    return _check(LIB.pf_eval_rhs(ctx, gamma, kphi, ku), ctx)


def pf_poisson_solve(ctx, rhs: int, x: int):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = LIB.pf_poisson_solve(ctx, rhs, x, ctypes.byref(it), ctypes.byref(rel))
    if st not in (PF_OK, PF_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return st, it.value, rel.value


def pf_sync(ctx):
    return _check(LIB.pf_sync(ctx), ctx)


def pf_destroy(ctx):
    LIB.pf_destroy(ctx)


def pf_profile_enable(ctx, enable: bool):
    return _check(LIB.pf_profile_enable(ctx, 1 if enable else 0), ctx)


def pf_profile_read(ctx, reset: bool = True) -> dict:
    """{kernel class: (launches, total ms)}"""
    arr = (pf_profile_entry * 32)()
    n = LIB.pf_profile_read(ctx, arr, 32, 1 if reset else 0)
    return {arr[i].name.decode(): (arr[i].launches, arr[i].ms) for i in range(min(n, 32))}


def pf_poisson_solve_static(params: pf_params, phi: int, rhs: int, x: int, stream: int | None):
    """Allocation-free solve (device pointers); returns (status, iterations, relres)."""
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = LIB.pf_poisson_solve_static(ctypes.byref(params), phi, rhs, x, stream, ctypes.byref(it),
                                     ctypes.byref(rel))
    if st not in (PF_OK, PF_ERR_NOT_CONVERGED):
        _check(st, None)
    return st, it.value, rel.value


def _params_array(plist):
    arr = (pf_params * len(plist))()
    for i, p in enumerate(plist):
        arr[i] = p
    return arr


def _check_batch(status, b=None):
    if status != PF_OK:
        msg = LIB.pf_batch_last_error(b)
        raise PFError(status, msg.decode() if msg else "")
    return status


def pf_batch_workspace_size(plist) -> int:
    n = ctypes.c_size_t(0)
    _check_batch(LIB.pf_batch_workspace_size(_params_array(plist), len(plist), ctypes.byref(n)))
    return n.value


def pf_batch_init(plist, workspace: int, workspace_bytes: int, nthreads: int = 0):
    b = ctypes.c_void_p(0)
    _check_batch(LIB.pf_batch_init(_params_array(plist), len(plist), workspace, workspace_bytes,
                                   nthreads, ctypes.byref(b)))
    return b


def pf_batch_step(b, nsteps: int):
    return _check_batch(LIB.pf_batch_step(b, nsteps), b)


def pf_batch_step_each(b, nsteps):
    arr = (ctypes.c_int * len(nsteps))(*[int(v) for v in nsteps])
    return _check_batch(LIB.pf_batch_step_each(b, arr), b)


def pf_batch_size(b) -> int:
    return LIB.pf_batch_size(b)


def pf_batch_context(b, i: int):
    return ctypes.c_void_p(LIB.pf_batch_context(b, i))


def pf_batch_destroy(b):
    LIB.pf_batch_destroy(b)


def pf_adjoint_workspace_size(params: pf_params) -> int:
    n = ctypes.c_size_t(0)
    _check(LIB.pf_adjoint_workspace_size(ctypes.byref(params), ctypes.byref(n)))
    return n.value


def pf_step_adjoint(ctx, workspace: int, workspace_bytes: int, state_n: int, lam: int,
                    gparam: int | None):
    return _check(LIB.pf_step_adjoint(ctx, workspace, workspace_bytes, state_n, lam, gparam), ctx)


def pf_objective(ctx, phi_target: int | None, w_ke: float, w_shape: float, grad: int,
                 gparam: int | None) -> float:
    J = ctypes.c_double(0.0)
    _check(LIB.pf_objective(ctx, phi_target, w_ke, w_shape, ctypes.byref(J), grad, gparam), ctx)
    return J.value


def pf_last_error(ctx=None) -> str:
    m = LIB.pf_last_error(ctx)
    return m.decode() if m else ""
