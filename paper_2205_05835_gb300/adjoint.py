"""Gradients of final-time objectives through many pf_step calls.

The reverse sweep runs in libpf (pf_step_adjoint: the transposed Jacobian of
one float64 step, recomputed from the step's initial state; pf_objective: the
objective and its gradient). This module only keeps the checkpoint schedule:
the forward pass stores the state every `every` steps, and the backward pass
walks the segments from the last to the first, recomputes the states inside
a segment from its checkpoint and applies the step transposes in reverse.

`Trajectory` and `Objective` wrap the two halves as torch.autograd.Function
so that a final-time objective of a run can be differentiated with
loss.backward() with respect to the initial phase field and the physical
parameters theta = (sigma, rho_in, rho_out, mu_in, mu_out).
"""
from __future__ import annotations

import torch

from . import binding as B

PARAM_NAMES = ("sigma", "rho_in", "rho_out", "mu_in", "mu_out")


def checkpoint_segments(nsteps: int, every: int):
    """[(first step, number of steps)] of the checkpoint segments, in forward order."""
    if nsteps < 0 or every < 1:
        raise ValueError("nsteps must be >= 0 and every >= 1")
    return [(s, min(every, nsteps - s)) for s in range(0, nsteps, every)]


class Adjoint:
    """The adjoint workspace of one Simulation (device memory owned by torch)."""

    def __init__(self, sim):
        self.sim = sim
        self.nbytes = B.pf_adjoint_workspace_size(sim.prm)
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8,
                                     device=sim.workspace.device)
        self.base = (self.workspace.data_ptr() + 255) // 256 * 256
        self.nvec = (1 + sim.dim) * sim.ncell

    def new_vector(self):
        return torch.zeros(self.nvec, dtype=torch.float64, device=self.workspace.device)

    def step(self, state_n, lam, gparam=None):
        """lam <- (d step / d state_n)^T lam; gparam += dJ/dtheta of the step."""
        assert lam.dtype == torch.float64 and lam.is_contiguous() and lam.numel() == self.nvec
        B.pf_step_adjoint(self.sim.ctx, self.base, self.nbytes, state_n.data_ptr(),
                          lam.data_ptr(), None if gparam is None else gparam.data_ptr())

    def objective(self, phi_target=None, w_ke=1.0, w_shape=0.0, gparam=None):
        """J of the simulation's current state and dJ/d(phi, u) (new tensor)."""
        grad = self.new_vector()
        tgt = None
        if phi_target is not None:
            assert phi_target.dtype == torch.float64 and phi_target.is_contiguous()
            tgt = phi_target.data_ptr()
        J = B.pf_objective(self.sim.ctx, tgt, float(w_ke), float(w_shape), grad.data_ptr(),
                           None if gparam is None else gparam.data_ptr())
        return J, grad


def forward_with_checkpoints(sim, nsteps: int, every: int):
    """Advance nsteps steps; returns the checkpoint states (device tensors)."""
    ckpts = []
    for first, count in checkpoint_segments(nsteps, every):
        ckpts.append(sim.state_tensor())
        sim.step(count)
    return ckpts


def backward_through(adj: Adjoint, ckpts, nsteps: int, every: int, lam, gparam):
    """lam: cotangent of the final state -> cotangent of the initial state."""
    sim = adj.sim
    segs = checkpoint_segments(nsteps, every)
    assert len(segs) == len(ckpts)
    for (first, count), ck in zip(reversed(segs), reversed(ckpts)):
        states = [ck]
        sim.load_state(ck)
        for _ in range(count - 1):
            sim.step(1)
            states.append(sim.state_tensor())
        for st in reversed(states):
            adj.step(st, lam, gparam)
    return lam


def set_initial(sim, phi0) -> None:
    """phi = phi0 (device or host float64), u = 0, p = 0."""
    z = torch.zeros(sim.ncell, dtype=torch.float64, device=sim.workspace.device)
    B.pf_set_field(sim.ctx, B.PF_FIELD_PHI, phi0.contiguous().reshape(-1).data_ptr())
    for f in (B.PF_FIELD_U, B.PF_FIELD_V) + ((B.PF_FIELD_W,) if sim.dim == 3 else ()):
        B.pf_set_field(sim.ctx, f, z.data_ptr())
    B.pf_set_field(sim.ctx, B.PF_FIELD_P, z.data_ptr())


def state_vector(sim):
    """(phi, u, v[, w]) of the current state as one float64 device vector."""
    out = torch.empty((1 + sim.dim) * sim.ncell, dtype=torch.float64,
                      device=sim.workspace.device)
    fields = [B.PF_FIELD_PHI, B.PF_FIELD_U, B.PF_FIELD_V, B.PF_FIELD_W][: 1 + sim.dim]
    for k, f in enumerate(fields):
        B.pf_get_field(sim.ctx, f, out[k * sim.ncell:(k + 1) * sim.ncell].data_ptr())
    return out


def _check_theta(sim, theta):
    vals = [float(v) for v in theta.detach().cpu().tolist()]
    want = [float(sim.params[k]) for k in PARAM_NAMES]
    if vals != want:
        raise ValueError(f"theta {vals} differs from the simulation's parameters {want}: "
                         "the gradient is taken at the simulation's parameters")


class Trajectory(torch.autograd.Function):
    """state_T = nsteps pf_step calls from (phi0, u = 0, p = 0).

    Inputs: phi0 (float64 device tensor shaped like the grid), theta (5
    float64 values equal to the simulation's sigma, rho_in, rho_out, mu_in,
    mu_out), the Simulation, nsteps and the checkpoint spacing. Output: the
    final (phi, u, v[, w]) as one float64 vector.
    """

    @staticmethod
    def forward(fctx, phi0, theta, sim, nsteps, every):
        _check_theta(sim, theta)
        set_initial(sim, phi0.detach())
        ckpts = forward_with_checkpoints(sim, nsteps, every)
        fctx.sim, fctx.nsteps, fctx.every, fctx.ckpts = sim, nsteps, every, ckpts
        fctx.phi_shape = phi0.shape
        return state_vector(sim)

    @staticmethod
    def backward(fctx, g_state):
        sim = fctx.sim
        adj = Adjoint(sim)
        lam = g_state.detach().to(torch.float64).contiguous().clone()
        gparam = torch.zeros(5, dtype=torch.float64, device=lam.device)
        backward_through(adj, fctx.ckpts, fctx.nsteps, fctx.every, lam, gparam)
        gphi0 = lam[: sim.ncell].reshape(fctx.phi_shape).clone()
        return gphi0, gparam, None, None, None


class Objective(torch.autograd.Function):
    """J = w_ke KE + (w_shape / 2) sum (phi - phi_target)^2 dV of a state vector."""

    @staticmethod
    def forward(fctx, state, theta, sim, phi_target, w_ke, w_shape):
        _check_theta(sim, theta)
        fields = [B.PF_FIELD_PHI, B.PF_FIELD_U, B.PF_FIELD_V, B.PF_FIELD_W][: 1 + sim.dim]
        st = state.detach().contiguous()
        for k, f in enumerate(fields):
            B.pf_set_field(sim.ctx, f, st[k * sim.ncell:(k + 1) * sim.ncell].data_ptr())
        adj = Adjoint(sim)
        gparam = torch.zeros(5, dtype=torch.float64, device=state.device)
        J, grad = adj.objective(phi_target, w_ke, w_shape, gparam)
        fctx.save_for_backward(grad, gparam)
        return torch.tensor(J, dtype=torch.float64, device=state.device)

    @staticmethod
    def backward(fctx, gJ):
        grad, gparam = fctx.saved_tensors
        return gJ * grad, gJ * gparam, None, None, None, None


def gradient(sim, phi0, nsteps, every, phi_target=None, w_ke=1.0, w_shape=0.0):
    """J and its gradient with respect to phi0 and theta (no autograd graph)."""
    set_initial(sim, phi0)
    ckpts = forward_with_checkpoints(sim, nsteps, every)
    adj = Adjoint(sim)
    gparam = torch.zeros(5, dtype=torch.float64, device=adj.workspace.device)
    J, lam = adj.objective(phi_target, w_ke, w_shape, gparam)
    backward_through(adj, ckpts, nsteps, every, lam, gparam)
    return J, lam[: sim.ncell].reshape(phi0.shape).clone(), gparam
