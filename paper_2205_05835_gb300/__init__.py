"""GB300-native phase-field two-phase flow step (energy-based surface tension).

The computation lives in libpf.so (CUDA, sm_103a) behind the C ABI of
include/pf.h; `binding` marshals arguments to it with ctypes, and
`Simulation` is a thin owner of the device workspace (allocated with torch)
and of one pf_ctx. There is no CPU fallback: importing the package raises if
the library is missing.
"""
from __future__ import annotations

import numpy as np

from . import binding as B
from .binding import (PFError, pf_batch_context, pf_batch_destroy, pf_batch_init,  # noqa: F401
                      pf_batch_size, pf_batch_step, pf_batch_workspace_size,
                      pf_destroy, pf_diagnostics, pf_eval_rhs, pf_get_field,
                      pf_get_state, pf_init, pf_last_error, pf_poisson_solve,
                      pf_profile_enable, pf_profile_read, pf_project,
                      pf_set_field, pf_set_state, pf_state_bytes, pf_step, pf_sync,
                      pf_workspace_size)

MODELS = {"cdi": 0, "sb": 1, "isodi": 2, "acdi": 3}
FORCES = {"eb": 0, "csf": 1, "lcsf": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
SCHEMES = {"rk4": 0, "fe": 1}
MOMENTUM = {"advective": 0, "consistent": 1}
SHAPES = {"drop": 0, "wave": 1}
FIELDS = {"phi": B.PF_FIELD_PHI, "u": B.PF_FIELD_U, "v": B.PF_FIELD_V, "w": B.PF_FIELD_W,
          "p": B.PF_FIELD_P}


def make_params(p: dict) -> B.pf_params:
    """pf_params from a dict (string names accepted for the enumerations)."""
    q = B.pf_params()
    q.dim = int(p["dim"])
    n = list(p["n"]) + [1] * (3 - len(p["n"]))
    for d in range(3):
        q.n[d] = int(n[d]) if (d < q.dim) else 1
    q.L = float(p.get("L", 1.0))

    def enum(key, table):
        v = p.get(key, 0)
        return table[v] if isinstance(v, str) else int(v)

    q.model = enum("model", MODELS)
    q.force = enum("force", FORCES)
    q.precision = enum("precision", PRECISIONS)
    q.scheme = enum("scheme", SCHEMES)
    q.momentum = enum("momentum", MOMENTUM)
    q.shape = enum("shape", SHAPES)
    for k in ("sigma", "eps", "rho_in", "rho_out", "mu_in", "mu_out", "gamma_fixed", "gamma_min",
              "dt", "delta_n", "poisson_rtol", "R", "pert_amp", "bound_tol", "inner_tol"):
        setattr(q, k, float(p.get(k, 0.0) or 0.0))
    for k in ("poisson_maxit", "pert_mode", "mg_pre", "mg_post", "use_graph", "wall_y",
              "mg_coarse_cells", "sweep_staging", "stage_kernel", "sweep_tile"):
        setattr(q, k, int(p.get(k, 0) or 0))
    return q


class Simulation:
    """One pf_ctx with its workspace on the current CUDA device (torch-owned)."""

    def __init__(self, params: dict, phi0=None, stream=None):
        import torch

        self.params = dict(params)
        self.prm = make_params(params)
        self.n = tuple(int(v) for v in self.prm.n)
        self.dim = self.prm.dim
        self.ncell = int(np.prod([self.n[d] for d in range(self.dim)]))
        self.shape = tuple(reversed([self.n[d] for d in range(self.dim)]))
        self.nbytes = pf_workspace_size(self.prm)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        base = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        ptr0 = None
        self._phi0_keep = None
        if phi0 is not None:
            t = torch.as_tensor(np.ascontiguousarray(phi0, dtype=np.float64)).reshape(-1)
            t = t.to(dev)
            self._phi0_keep = t
            ptr0 = t.data_ptr()
        self.ctx = pf_init(self.prm, base, self.nbytes, ptr0, self.stream.cuda_stream)
        self._phi0_keep = None

    def step(self, nsteps=1):
        pf_step(self.ctx, nsteps)

    def project(self):
        pf_project(self.ctx)

    def diagnostics(self) -> dict:
        return pf_diagnostics(self.ctx)

    def field(self, name: str) -> np.ndarray:
        out = np.empty(self.ncell, dtype=np.float64)
        pf_get_field(self.ctx, FIELDS[name], out.ctypes.data)
        return out.reshape(self.shape)

    def set_field(self, name: str, values) -> None:
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(-1)
        assert a.size == self.ncell
        pf_set_field(self.ctx, FIELDS[name], a.ctypes.data)

    def velocity(self):
        return [self.field("uvw"[d]) for d in range(self.dim)]

    def eval_rhs(self, gamma: float):
        kphi = np.empty(self.ncell, dtype=np.float64)
        ku = np.empty(self.dim * self.ncell, dtype=np.float64)
        pf_eval_rhs(self.ctx, float(gamma), kphi.ctypes.data, ku.ctypes.data)
        return kphi.reshape(self.shape), [ku[d * self.ncell:(d + 1) * self.ncell].reshape(self.shape)
                                          for d in range(self.dim)]

    def poisson_solve(self, rhs, x0=None):
        r = np.ascontiguousarray(rhs, dtype=np.float64).reshape(-1)
        x = np.zeros(self.ncell) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).reshape(-1).copy()
        st, it, rel = pf_poisson_solve(self.ctx, r.ctypes.data, x.ctypes.data)
        return x.reshape(self.shape), it, rel, st

    def state_bytes(self) -> int:
        return pf_state_bytes(self.ctx)

    def state_tensor(self):
        """The raw state (pf_get_state layout) in a new device uint8 tensor."""
        import torch

        t = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.workspace.device)
        pf_get_state(self.ctx, t.data_ptr())
        return t

    def load_state(self, t) -> None:
        """Restore a state taken by state_tensor (host or device tensor)."""
        assert t.numel() == self.state_bytes() and t.is_contiguous()
        pf_set_state(self.ctx, t.data_ptr())

    def close(self):
        if getattr(self, "ctx", None) is not None:
            pf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent instances advanced together (pf_batch_*); workspace
    allocated with torch on the current device."""

    def __init__(self, param_list, nthreads=0):
        import torch

        self.params = [dict(p) for p in param_list]
        self.prms = [make_params(p) for p in param_list]
        self.nbytes = pf_batch_workspace_size(self.prms)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=dev)
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        self.b = pf_batch_init(self.prms, base, self.nbytes, nthreads)
        self.cells = [int(np.prod([p.n[d] for d in range(p.dim)])) for p in self.prms]

    def __len__(self):
        return len(self.prms)

    def step(self, nsteps=1):
        pf_batch_step(self.b, nsteps)

    def step_each(self, nsteps):
        """Instance i advances nsteps[i] steps."""
        B.pf_batch_step_each(self.b, nsteps)

    def field(self, i, name):
        p = self.prms[i]
        shape = tuple(reversed([p.n[d] for d in range(p.dim)]))
        out = np.empty(self.cells[i], dtype=np.float64)
        pf_get_field(pf_batch_context(self.b, i), FIELDS[name], out.ctypes.data)
        return out.reshape(shape)

    def diagnostics(self, i):
        return pf_diagnostics(pf_batch_context(self.b, i))

    def close(self):
        if getattr(self, "b", None) is not None:
            pf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
