"""Consistent (conservative) momentum transport on the GPU (momentum = 1).

Parity with the FP64 oracle (right-hand side to 1e-12, whole steps to 1e-10),
the two properties that define the transport checked on the GPU's own output
(exact conservation of sum rho_f u without surface tension; a uniform velocity
carried unchanged through a moving density field), the mixed path's per-field
distance from the float64 path, and graph mode."""
import numpy as np
import pytest

import pf_inputs as I
from oracle import pf_oracle as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def pf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2205_05835_gb300 as pf

    return pf


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def case(dim, n, **kw):
    base = dict(momentum="consistent", rho_in=1000.0, rho_out=1.0, mu_in=0.05, mu_out=0.002,
                poisson_rtol=1e-13, poisson_maxit=400)
    base.update(kw)
    return I.small_case(dim=dim, n=n, **base)


@pytest.mark.parametrize("dim,n", [(2, (40, 40, 1)), (3, (24, 20, 16))])
def test_consistent_rhs_parity(pf, dim, n):
    p = case(dim, n[0])
    p["n"] = n
    po = O.params_from(p)
    g = O.Grid(dim, n, p["L"])
    phi = O.initial_phi(po) + 0.02 * (I.noise(g.shape, 3) - 0.5)
    u = [0.3 * (I.noise(g.shape, 4 + d) - 0.5) for d in range(dim)]
    sim = pf.Simulation(p, phi0=phi)
    for d in range(dim):
        sim.set_field("uvw"[d], u[d])
    gam = 0.37
    kphi, ku = sim.eval_rhs(gam)
    want = O.momentum_rhs_consistent(phi, u, g, po, gam)
    assert rel(kphi, O.phase_rhs(phi, u, g, po, gam)) < 1e-12
    for d in range(dim):
        assert rel(ku[d], want[d]) < 1e-12, d
    sim.close()


@pytest.mark.parametrize("dim,n,scheme,steps", [(2, 64, "rk4", 3), (2, 48, "fe", 4),
                                                (3, 16, "rk4", 2)])
def test_consistent_step_parity_fp64(pf, dim, n, scheme, steps):
    p = case(dim, n, scheme=scheme, gamma_fixed=0.3)
    po = O.params_from(p)
    st = O.run(po, steps=steps)
    sim = pf.Simulation(p)
    sim.step(steps)
    assert rel(sim.field("phi"), st.phi) < TOL64
    for d in range(dim):
        assert rel(sim.field("uvw"[d]), st.u[d]) < TOL64, d
    assert rel(sim.field("p"), st.p - st.p.mean()) < TOL64
    sim.close()


def total_momentum(phi, u, g, po):
    rf = O.face_density(phi, g, po)
    return np.array([float(np.sum(rf[d] * u[d])) for d in range(g.dim)])


def test_consistent_momentum_conserved_on_gpu(pf):
    """Exact for any pressure: the projection changes sum rho_f u by -tau sum G p,
    a telescoping sum (so the solve tolerance does not enter)."""
    p = case(2, 48, sigma=0.0, gamma_fixed=0.5, dt=1e-4, poisson_rtol=1e-11)
    po = O.params_from(p)
    g = O.Grid(2, p["n"], p["L"])
    sim = pf.Simulation(p)
    u0 = [0.2 * (I.noise(g.shape, 11 + d) - 0.5) for d in range(2)]
    for d in range(2):
        sim.set_field("uv"[d], u0[d])
    sim.project()
    P0 = total_momentum(sim.field("phi"), [sim.field("u"), sim.field("v")], g, po)
    sim.step(5)
    phi = sim.field("phi")
    assert 0.0 < phi.min() and phi.max() < 1.0
    P1 = total_momentum(phi, [sim.field("u"), sim.field("v")], g, po)
    scale = float(np.sum(O.density_cells(phi, po))) * 0.2
    assert np.max(np.abs(P1 - P0)) < 1e-12 * scale, (P0, P1)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_consistent_uniform_velocity_preserved(pf, precision):
    p = case(2, 48, sigma=0.0, gamma_fixed=0.5, dt=1e-4, pert_amp=0.2, precision=precision,
             poisson_rtol=1e-10)
    sim = pf.Simulation(p)
    U, V = 0.3, -0.2
    shape = (48, 48)
    sim.set_field("u", np.full(shape, U))
    sim.set_field("v", np.full(shape, V))
    sim.step(4)
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert np.max(np.abs(sim.field("u") - U)) < tol
    assert np.max(np.abs(sim.field("v") - V)) < tol
    sim.close()


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 32)])
def test_consistent_mixed_per_field_error(pf, dim, n):
    """Mixed precision (float32 stencils, double-float pressure) against the
    float64 GPU path after three steps of a density-ratio-1000 drop: stated
    bounds phi < 1e-5, u < 1e-2, p < 1e-3 (max-norm relative)."""
    p64 = case(dim, n, poisson_rtol=1e-12)
    p32 = dict(p64, precision="mixed", poisson_rtol=1e-10)
    a = pf.Simulation(p64)
    b = pf.Simulation(p32)
    a.step(3)
    b.step(3)
    names = ("phi", "u", "v", "w", "p")[: dim + 1] if dim == 3 else ("phi", "u", "v")
    errs = {c: rel(b.field(c), a.field(c)) for c in names + ("p",)}
    assert errs["phi"] < 1e-5, errs
    assert max(errs[c] for c in names[1:]) < 1e-2, errs
    assert errs["p"] < 1e-3, errs
    a.close()
    b.close()


def test_consistent_graph_mode_matches(pf):
    p = case(3, 16, precision="mixed", poisson_rtol=1e-10)
    a = pf.Simulation(p)
    b = pf.Simulation(dict(p, use_graph=1))
    a.step(3)
    b.step(3)
    for c in ("phi", "u", "v", "w", "p"):
        np.testing.assert_array_equal(a.field(c), b.field(c))
    a.close()
    b.close()
