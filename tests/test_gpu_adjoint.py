"""Reverse mode of the float64 step (pf_step_adjoint, pf_objective) through the C ABI.

The reference derivatives come from the oracle, never from the CUDA path:
  * one step: the dot-product identity <w, J v> = <J^T w, v>, with J v from the
    oracle by the complex-step method (step evaluated at X + i h v, h = 1e-30,
    J v = Im / h: exact to rounding, no cancellation), for the state and for
    each parameter sigma, rho_in, rho_out, mu_in, mu_out;
  * Gamma tracked as max |u^n|: the oracle's central difference (|u| is not
    analytic, so no complex step);
  * many steps with checkpoints: the objective's directional derivative along
    a seeded direction of phi0 (complex step) and its sigma derivative
    (the oracle's central difference, h = 1e-6);
  * the 256^2 differentiable oscillating drop (500 steps, checkpoint every 25):
    central differences h = 1e-6 of the GPU forward run.
Phi stays strictly inside (0, 1) in every case (clip is differentiable there).
"""
import numpy as np
import pytest

import pf_inputs as I
from oracle import pf_oracle as O

pytestmark = pytest.mark.gpu

PARAMS = ("sigma", "rho_in", "rho_out", "mu_in", "mu_out")
HC = 1e-30   # complex step


@pytest.fixture(scope="module")
def pf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2205_05835_gb300 as pf

    return pf


def case(dim, n, scheme, **kw):
    base = dict(scheme=scheme, gamma_fixed=0.05, poisson_rtol=1e-13, mu_out=0.004)
    base.update(kw)
    return I.small_case(dim=dim, n=n, **base)


def start_state(p, seed):
    """Perturbed drop (phi strictly inside (0, 1)) and a seeded velocity."""
    po = O.params_from(p)
    g = O.Grid(p["dim"], p["n"], p["L"])
    phi0 = O.initial_phi(po)
    phi = phi0 + 0.1 * phi0 * (1.0 - phi0) * (I.noise(g.shape, seed) - 0.5)
    u = [0.05 * (I.noise(g.shape, seed + 1 + d) - 0.5) for d in range(g.dim)]
    return g, phi, u


def load(sim, phi, u):
    sim.set_field("phi", phi)
    for d, c in enumerate("uvw"[: len(u)]):
        sim.set_field(c, u[d])
    sim.set_field("p", np.zeros_like(phi))


def flat(phi, u):
    return np.concatenate([phi.ravel()] + [c.ravel() for c in u])


def oracle_step(phi, u, p):
    st = O.State(phi, list(u), np.zeros(phi.shape, dtype=phi.dtype))
    out = O.step(st, p)
    return out.phi, out.u


def vjp_gpu(pf, sim, w):
    import torch

    from paper_2205_05835_gb300 import adjoint as A

    adj = A.Adjoint(sim)
    state = sim.state_tensor()
    lam = torch.tensor(w, dtype=torch.float64, device="cuda")
    gp = torch.zeros(5, dtype=torch.float64, device="cuda")
    adj.step(state, lam, gp)
    return lam.cpu().numpy(), gp.cpu().numpy()


@pytest.mark.parametrize("scheme", ["fe", "rk4"])
@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16)])
def test_step_transpose_matches_complex_step(pf, scheme, dim, n):
    p = case(dim, n, scheme)
    po = O.params_from(p)
    g, phi, u = start_state(p, 100 + dim)
    N = phi.size
    assert 0.0 < phi.min() and phi.max() < 1.0
    sim = pf.Simulation(p)
    load(sim, phi, u)
    w = I.noise((1 + dim) * N, 7) - 0.5
    v = I.noise((1 + dim) * N, 8) - 0.5
    lam, gp = vjp_gpu(pf, sim, w)
    # J v of the oracle by the complex step
    vphi = v[:N].reshape(g.shape)
    vu = [v[(1 + d) * N:(2 + d) * N].reshape(g.shape) for d in range(dim)]
    ph1, u1 = oracle_step(phi + 1j * HC * vphi, [u[d] + 1j * HC * vu[d] for d in range(dim)], po)
    # clip(phi) is differentiated everywhere except exactly at 0 and 1
    assert not np.any((ph1.real == 0.0) | (ph1.real == 1.0))
    jv = flat(ph1.imag, [c.imag for c in u1]) / HC
    lhs, rhs = float(w @ jv), float(lam @ v)
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + np.linalg.norm(w) * np.linalg.norm(jv) * 1e-3), (lhs, rhs)
    # parameters
    for k, name in enumerate(PARAMS):
        q = dict(po)
        q[name] = q[name] + 1j * HC
        ph1, u1 = oracle_step(phi.astype(complex), [c.astype(complex) for c in u], q)
        d_theta = float(w @ flat(ph1.imag, [c.imag for c in u1])) / HC
        scale = abs(d_theta) + 1e-12 * np.linalg.norm(w)
        assert abs(gp[k] - d_theta) <= 1e-9 * scale + 1e-14, (name, gp[k], d_theta)
    sim.close()


@pytest.mark.parametrize("scheme", ["fe", "rk4"])
def test_step_transpose_tracked_gamma(pf, scheme):
    """Gamma = max |u^n|: the derivative goes to the maximising face."""
    p = case(2, 32, scheme, gamma_fixed=0.0, gamma_min=0.0)
    po = O.params_from(p)
    g, phi, u = start_state(p, 300)
    N = phi.size
    sim = pf.Simulation(p)
    load(sim, phi, u)
    w = I.noise(3 * N, 17) - 0.5
    v = I.noise(3 * N, 18) - 0.5
    v[:N] *= (phi * (1.0 - phi)).ravel()   # real differences must not cross clip's kinks
    lam, _ = vjp_gpu(pf, sim, w)
    h = 1e-6

    def J(s):
        ph1, u1 = oracle_step(phi + s * v[:N].reshape(g.shape),
                              [u[d] + s * v[(1 + d) * N:(2 + d) * N].reshape(g.shape)
                               for d in range(2)], po)
        return float(w @ flat(ph1, u1))

    fd = (J(h) - J(-h)) / (2 * h)
    got = float(lam @ v)
    assert abs(got - fd) <= 1e-6 * abs(fd), (got, fd)
    # with Gamma frozen at the same value, the transpose differs at exactly one
    # entry: the face where |u^n| is largest
    umax = max(float(np.max(np.abs(c))) for c in u)
    p2 = dict(p, gamma_fixed=umax)
    sim2 = pf.Simulation(p2)
    load(sim2, phi, u)
    lam2, _ = vjp_gpu(pf, sim2, w)
    diff = np.nonzero(lam - lam2)[0]
    k = int(np.argmax(np.abs(flat(np.zeros_like(phi), u))))
    assert list(diff) == [k], (diff[:5], k)
    sim.close()
    sim2.close()


def oracle_objective(st, po, target, w_ke, w_shape):
    """w_ke KE + (w_shape / 2) sum (phi - target)^2 dV (complex-safe)."""
    g = O.Grid(po["dim"], po["n"], po["L"])
    rho = O.density_cells(st.phi, po)
    ke = 0.0
    for d in range(g.dim):
        ke = ke + 0.5 * np.sum(O.face_avg(rho, g, d) * st.u[d] ** 2) * g.dV
    return w_ke * ke + 0.5 * w_shape * np.sum((st.phi - target) ** 2) * g.dV


def oracle_run_J(phi0, po, steps, target, w_ke, w_shape):
    g = O.Grid(po["dim"], po["n"], po["L"])
    st = O.State(phi0, [np.zeros(g.shape, dtype=phi0.dtype) for _ in range(g.dim)],
                 np.zeros(g.shape, dtype=phi0.dtype))
    for _ in range(steps):
        st = O.step(st, po)
    return oracle_objective(st, po, target, w_ke, w_shape)


@pytest.mark.parametrize("scheme,steps,every", [("rk4", 10, 4), ("fe", 12, 5)])
def test_trajectory_gradient_vs_oracle(pf, scheme, steps, every):
    import torch

    from paper_2205_05835_gb300 import adjoint as A

    p = case(2, 32, scheme)
    po = O.params_from(p)
    g = O.Grid(2, p["n"], p["L"])
    phi0 = O.initial_phi(po)
    target = O.initial_phi(dict(po, pert_amp=0.0))
    w_ke, w_shape = 1.0, 10.0
    sim = pf.Simulation(p)
    J, gphi, gp = A.gradient(sim, torch.tensor(phi0, device="cuda"), steps, every,
                             torch.tensor(target, device="cuda"), w_ke, w_shape)
    gphi, gp = gphi.cpu().numpy(), gp.cpu().numpy()
    J_or = oracle_run_J(phi0, po, steps, target, w_ke, w_shape)
    assert abs(J - J_or) <= 1e-10 * abs(J_or)
    # direction of phi0 that keeps phi inside (0, 1)
    v = phi0 * (1 - phi0) * (I.noise(g.shape, 21) - 0.5)
    d_or = oracle_run_J(phi0 + 1j * HC * v, po, steps, target, w_ke, w_shape).imag / HC
    d_gpu = float(np.sum(gphi * v))
    assert abs(d_gpu - d_or) <= 1e-9 * abs(d_or), (d_gpu, d_or)
    # sigma: the oracle's own central difference
    h = 1e-6
    Jp = oracle_run_J(phi0, dict(po, sigma=po["sigma"] + h), steps, target, w_ke, w_shape)
    Jm = oracle_run_J(phi0, dict(po, sigma=po["sigma"] - h), steps, target, w_ke, w_shape)
    fd = (Jp - Jm) / (2 * h)
    assert abs(gp[0] - fd) <= 1e-6 * abs(fd), (gp[0], fd)
    # rho_in and mu_in by complex step
    for k, name in ((1, "rho_in"), (3, "mu_in")):
        q = dict(po)
        q[name] = q[name] + 1j * HC
        d = oracle_run_J(phi0.astype(complex), q, steps, target, w_ke, w_shape).imag / HC
        assert abs(gp[k] - d) <= 1e-9 * abs(d) + 1e-16, (name, gp[k], d)
    sim.close()


def test_autograd_function_matches_direct(pf):
    import torch

    from paper_2205_05835_gb300 import adjoint as A

    p = case(2, 32, "rk4")
    po = O.params_from(p)
    phi0 = torch.tensor(O.initial_phi(po), device="cuda", requires_grad=True)
    theta = torch.tensor([p[k] for k in PARAMS], dtype=torch.float64, device="cuda",
                         requires_grad=True)
    target = torch.tensor(O.initial_phi(dict(po, pert_amp=0.0)), device="cuda")
    sim = pf.Simulation(p)
    state = A.Trajectory.apply(phi0, theta, sim, 8, 3)
    J = A.Objective.apply(state, theta, sim, target, 1.0, 5.0)
    J.backward()
    sim2 = pf.Simulation(p)
    J2, g2, gp2 = A.gradient(sim2, phi0.detach(), 8, 3, target, 1.0, 5.0)
    assert abs(J.item() - J2) <= 1e-13 * abs(J2)
    assert torch.allclose(phi0.grad, g2, rtol=0, atol=1e-12 * float(g2.abs().max()))
    assert torch.allclose(theta.grad, gp2, rtol=1e-12, atol=0)
    sim.close()
    sim2.close()


def test_oscillating_drop_256_fd(pf):
    """256^2 mode-2 drop, density ratio 10, 500 RK4 steps, checkpoint every 25:
    adjoint vs central differences (h = 1e-6) of the GPU forward."""
    import torch

    from paper_2205_05835_gb300 import adjoint as A

    p = dict(I.oscillating_drop_2d_256(), gamma_fixed=0.1, poisson_rtol=1e-13)
    p = I.finalize(p)
    po = O.params_from(p)
    steps, every = p["steps"], 25
    phi0 = torch.tensor(O.initial_phi(po), device="cuda")
    target = torch.tensor(O.initial_phi(dict(po, pert_amp=0.0)), device="cuda")
    w_ke, w_shape = 1.0, 1.0
    sim = pf.Simulation(p)
    J, gphi, gp = A.gradient(sim, phi0, steps, every, target, w_ke, w_shape)

    def run(q, ph0):
        s = pf.Simulation(q)
        A.set_initial(s, ph0)
        s.step(steps)
        a = A.Adjoint(s)
        Jv, _ = a.objective(target, w_ke, w_shape)
        s.close()
        return Jv

    h = 1e-6
    fd_sigma = (run(dict(p, sigma=p["sigma"] + h), phi0) -
                run(dict(p, sigma=p["sigma"] - h), phi0)) / (2 * h)
    assert abs(gp[0].item() - fd_sigma) <= 1e-5 * abs(fd_sigma), (gp[0].item(), fd_sigma)
    v = phi0 * (1 - phi0) * torch.tensor(I.noise(tuple(phi0.shape), 31) - 0.5, device="cuda")
    fd_phi = (run(p, phi0 + h * v) - run(p, phi0 - h * v)) / (2 * h)
    got = float((gphi * v).sum())
    assert abs(got - fd_phi) <= 1e-5 * abs(fd_phi), (got, fd_phi)
    sim.close()
