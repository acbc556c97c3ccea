"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Float64 path: fields within 1e-10 relative (max |gpu - oracle| / max |oracle|)
of the oracle; the CG solves are run to a relative residual the oracle's exact
solve can be compared with. Mixed path: per-field bounds stated in each test.
"""
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


def rand_velocity(g, seed, amp=0.3):
    """Seeded face velocity (not divergence free) for operator tests."""
    return [amp * (I.noise(g.shape, seed + d) - 0.5) for d in range(g.dim)]


# --------------------------------------------------------------------------
# initial condition
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n,mode", [(2, 40, 2), (2, 33, 0), (3, 24, 2), (3, 20, 3)])
def test_init_profile(pf, dim, n, mode):
    p = I.small_case(dim=dim, n=n, pert_mode=mode, pert_amp=0.05 if mode else 0.0)
    sim = pf.Simulation(p)
    want = O.initial_phi(O.params_from(p))
    assert np.max(np.abs(sim.field("phi") - want)) < 1e-14
    for c in "uvw"[:dim]:
        assert np.max(np.abs(sim.field(c))) == 0.0
    sim.close()


# --------------------------------------------------------------------------
# operator parity: phase-field and momentum right-hand sides
# --------------------------------------------------------------------------
CASES = [(m, f) for m in ("cdi", "sb", "isodi", "acdi") for f in ("eb", "csf", "lcsf")]


@pytest.mark.parametrize("model,force", CASES)
@pytest.mark.parametrize("dim,n", [(2, (40, 40, 1)), (3, (24, 20, 16))])
def test_rhs_parity_fp64(pf, model, force, dim, n):
    p = I.small_case(dim=dim, n=n[0], model=model, force=force)
    p["n"] = n
    po = O.params_from(p)
    g = O.Grid(dim, n, p["L"])
    phi = O.initial_phi(po) + 0.02 * (I.noise(g.shape, 7) - 0.5)
    u = rand_velocity(g, 11)
    sim = pf.Simulation(p, phi0=phi)
    for d in range(dim):
        sim.set_field("uvw"[d], u[d])
    gam = 0.37
    kphi, ku = sim.eval_rhs(gam)
    want_phi = O.phase_rhs(phi, u, g, po, gam)
    want_u = O.momentum_rhs(phi, u, g, po)
    assert rel(kphi, want_phi) < 1e-12
    for d in range(dim):
        assert rel(ku[d], want_u[d]) < 1e-12, d
    sim.close()


@pytest.mark.parametrize("model,force", [("cdi", "eb"), ("isodi", "lcsf"), ("sb", "csf"),
                                         ("acdi", "eb"), ("acdi", "csf")])
def test_rhs_parity_mixed(pf, model, force):
    """float32 stencils: relative to the field scale, within 2e-5 (phase field) and
    1e-4 (momentum, where the force is a difference of O(1/eps) terms)."""
    p = I.small_case(dim=3, n=24, model=model, force=force, precision="mixed")
    po = O.params_from(p)
    g = O.Grid(3, p["n"], p["L"])
    phi = O.initial_phi(po)
    u = rand_velocity(g, 3, amp=0.1)
    sim = pf.Simulation(p, phi0=phi)
    for d in range(3):
        sim.set_field("uvw"[d], u[d])
    # the mixed path stores phi and u in float32: compare with the oracle on the
    # rounded inputs
    phi32 = phi.astype(np.float32).astype(np.float64)
    u32 = [c.astype(np.float32).astype(np.float64) for c in u]
    kphi, ku = sim.eval_rhs(0.2)
    assert rel(kphi, O.phase_rhs(phi32, u32, g, po, 0.2)) < 2e-5
    want_u = O.momentum_rhs(phi32, u32, g, po)
    for d in range(3):
        assert rel(ku[d], want_u[d]) < 1e-4
    sim.close()


# --------------------------------------------------------------------------
# Poisson solve
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n,ratio", [(2, (48, 48, 1), 1000.0), (2, (40, 40, 1), 10.0),
                                         (3, (16, 16, 16), 100.0), (3, (24, 20, 16), 10.0)])
def test_poisson_solve_fp64(pf, dim, n, ratio):
    p = I.small_case(dim=dim, n=n[0], rho_in=ratio, rho_out=1.0, poisson_rtol=1e-13,
                     poisson_maxit=400)
    p["n"] = n
    po = O.params_from(p)
    g = O.Grid(dim, n, p["L"])
    phi = O.initial_phi(po)
    rhs = I.noise(g.shape, 5) - 0.5
    rhs -= rhs.mean()
    sim = pf.Simulation(p, phi0=phi)
    x, it, relres, st = sim.poisson_solve(rhs)
    assert st == 0, pf.pf_last_error(sim.ctx)
    assert relres <= 1e-13
    beta = O.face_beta(phi, g, po)
    want = O.solve_poisson(beta, rhs, g)
    assert rel(x, want) < 1e-9
    res = O.apply_poisson(beta, x, g) - rhs
    assert np.linalg.norm(res) <= 2e-13 * np.linalg.norm(rhs)
    sim.close()


def beta_f32(phi, g, p):
    """Face coefficients of the mixed-precision operator: 1 / rho_f evaluated and
    rounded in float32 (phi stored in float32), promoted to float64."""
    ph = phi.astype(np.float32)
    c = np.clip(ph, np.float32(0), np.float32(1))
    dr = np.float32(np.float32(p["rho_in"]) - np.float32(p["rho_out"]))
    rho = np.float32(p["rho_out"]) + (dr * c).astype(np.float32)
    out = []
    for d in range(g.dim):
        rf = np.float32(0.5) * (rho + np.roll(rho, 1, axis=g.axis(d)))
        out.append((np.float32(1) / rf).astype(np.float64))
    return out


def test_poisson_mixed_preconditioner_reaches_fp64_residual(pf):
    """float32 inner solves inside float64 iterative refinement reach a 1e-12
    float64 residual of the mixed operator (float32-rounded face coefficients)."""
    p = I.small_case(dim=3, n=32, rho_in=10.0, rho_out=1.0, precision="mixed",
                     poisson_rtol=1e-12, poisson_maxit=200)
    po = O.params_from(p)
    g = O.Grid(3, p["n"], p["L"])
    phi = O.initial_phi(po)
    rhs = I.noise(g.shape, 9) - 0.5
    rhs -= rhs.mean()
    sim = pf.Simulation(p, phi0=phi)
    x, it, relres, st = sim.poisson_solve(rhs)
    assert st == 0 and relres <= 1e-12
    res = O.apply_poisson(beta_f32(phi, g, po), x, g) - rhs
    assert np.linalg.norm(res) <= 2e-12 * np.linalg.norm(rhs)
    # and it solves the float64 operator to float32 accuracy of its coefficients
    phi32 = phi.astype(np.float32).astype(np.float64)
    res64 = O.apply_poisson(O.face_beta(phi32, g, po), x, g) - rhs
    assert np.linalg.norm(res64) <= 1e-6 * np.linalg.norm(rhs)
    sim.close()


def test_poisson_iteration_cap_reports_not_converged(pf):
    p = I.small_case(dim=2, n=32, poisson_rtol=1e-14, poisson_maxit=1)
    po = O.params_from(p)
    g = O.Grid(2, p["n"], p["L"])
    sim = pf.Simulation(p)
    rhs = I.noise(g.shape, 1) - 0.5
    x, it, relres, st = sim.poisson_solve(rhs - rhs.mean())
    assert st == pf.B.PF_ERR_NOT_CONVERGED and it == 1
    # the context stays usable
    sim2 = pf.Simulation(dict(p, poisson_maxit=200))
    x, it, relres, st = sim2.poisson_solve(rhs - rhs.mean())
    assert st == 0
    sim.close()
    sim2.close()


# --------------------------------------------------------------------------
# whole steps
# --------------------------------------------------------------------------
def run_both(pf, p, steps):
    po = O.params_from(p)
    phi0 = O.initial_phi(po)
    sim = pf.Simulation(p, phi0=phi0)
    sim.step(steps)
    st = O.run(po, steps=steps, phi0=phi0)
    return sim, st


@pytest.mark.parametrize("model,force,scheme", [
    ("cdi", "eb", "rk4"), ("cdi", "csf", "rk4"), ("cdi", "lcsf", "rk4"),
    ("sb", "eb", "rk4"), ("isodi", "eb", "fe"), ("sb", "lcsf", "fe"),
    ("acdi", "eb", "rk4"), ("acdi", "lcsf", "fe")])
def test_step_parity_fp64_2d(pf, model, force, scheme):
    p = I.small_case(dim=2, n=40, model=model, force=force, scheme=scheme,
                     poisson_rtol=1e-13, poisson_maxit=300, gamma_min=0.05)
    sim, st = run_both(pf, p, 5)
    assert rel(sim.field("phi"), st.phi) < TOL64
    assert rel(sim.field("u"), st.u[0]) < TOL64
    assert rel(sim.field("v"), st.u[1]) < TOL64
    assert rel(sim.field("p"), st.p) < TOL64
    d = sim.diagnostics()
    od = O.diagnostics(st, p)
    for k in ("mass", "ke", "se", "umax", "phi_min", "phi_max", "dp_laplace"):
        assert abs(d[k] - od[k]) <= 1e-10 * max(abs(od[k]), 1e-30) + 1e-300, k
    sim.close()


@pytest.mark.parametrize("model,force", [("cdi", "eb"), ("cdi", "lcsf"), ("acdi", "eb")])
def test_step_parity_fp64_3d(pf, model, force):
    p = I.small_case(dim=3, n=16, model=model, force=force, poisson_rtol=1e-13, poisson_maxit=300)
    p["n"] = (16, 16, 16)
    sim, st = run_both(pf, p, 3)
    for name, ref in (("phi", st.phi), ("u", st.u[0]), ("v", st.u[1]), ("w", st.u[2]),
                      ("p", st.p)):
        assert rel(sim.field(name), ref) < TOL64, name
    sim.close()


def test_static_drop_64_fp64_200_steps(pf):
    """The 64^2 static drop (FP64, CDI + EB, La = 12000) over its 200 steps."""
    p = dict(I.static_drop_64(), poisson_rtol=1e-13, poisson_maxit=300)
    sim, st = run_both(pf, p, p["steps"])
    for name, ref in (("phi", st.phi), ("u", st.u[0]), ("v", st.u[1]), ("p", st.p)):
        assert rel(sim.field(name), ref) < TOL64, name
    d = sim.diagnostics()
    od = O.diagnostics(st, p)
    assert abs(d["ca_inf"] - od["ca_inf"]) <= 1e-10 * od["ca_inf"]
    assert abs(d["mass"] - od["mass"]) <= 1e-13 * od["mass"]
    assert d["poisson_relres"] <= 1e-13
    sim.close()


def test_step_mixed_per_field_error(pf):
    """Mixed precision vs the FP64 oracle after 5 RK4 steps (ratio-10 drop):
    phi within 1e-5, velocity within 2e-3 of its max, pressure within 1e-4."""
    p = I.small_case(dim=2, n=48, precision="mixed", poisson_rtol=1e-12)
    po = O.params_from(p)
    phi0 = O.initial_phi(po).astype(np.float32).astype(np.float64)
    sim = pf.Simulation(p, phi0=phi0)
    sim.step(5)
    st = O.run(dict(po, precision="fp64"), steps=5, phi0=phi0)
    assert rel(sim.field("phi"), st.phi) < 1e-5
    assert rel(sim.field("u"), st.u[0]) < 2e-3
    assert rel(sim.field("v"), st.u[1]) < 2e-3
    assert rel(sim.field("p"), st.p) < 1e-4
    sim.close()


def test_state_round_trip_and_restart(pf):
    """get_state / set_state restarts bit-identically (checkpoint/resume)."""
    p = I.small_case(dim=2, n=32, poisson_rtol=1e-13)
    a = pf.Simulation(p)
    a.step(2)
    buf = np.empty(a.state_bytes(), dtype=np.uint8)
    pf.pf_get_state(a.ctx, buf.ctypes.data)
    a.step(2)
    b = pf.Simulation(p)
    pf.pf_set_state(b.ctx, buf.ctypes.data)
    b.step(2)
    for name in ("phi", "u", "v", "p"):
        np.testing.assert_array_equal(a.field(name), b.field(name))
    assert a.diagnostics()["step"] == b.diagnostics()["step"] == 4
    a.close()
    b.close()


def test_nonfinite_input_is_reported(pf):
    p = I.small_case(dim=2, n=32)
    po = O.params_from(p)
    phi = O.initial_phi(po)
    phi[3, 5] = np.nan
    sim = pf.Simulation(p, phi0=phi)
    with pytest.raises(pf.PFError) as e:
        sim.diagnostics()
    assert e.value.status == pf.B.PF_ERR_NONFINITE
    sim.close()


@pytest.mark.parametrize("n", [(4, 4, 1), (6, 10, 1), (4, 4, 4), (12, 8, 6)])
def test_tiny_and_odd_grids(pf, n):
    dim = 2 if n[2] == 1 else 3
    p = I.small_case(dim=dim, n=n[0], poisson_rtol=1e-13, poisson_maxit=500, R=0.3)
    p["n"] = n
    sim, st = run_both(pf, p, 2)
    assert rel(sim.field("phi"), st.phi) < TOL64
    assert rel(sim.field("p"), st.p) < 1e-9
    sim.close()


@pytest.mark.parametrize("n", [(40, 40, 40), (48, 40, 24), (64, 64, 64), (42, 40, 24)])
def test_poisson_mixed_3d_sweeps_converge(pf, n):
    """3D float32 levels use the one-pass tiled red-black sweep (ragged tiles when a
    size is not a multiple of the 32 x 8 tile): the refined solve still reaches a
    1e-12 float64 residual of the float32 operator in few inner iterations (a
    faulty smoother still converges inside flexible CG, only more slowly: about
    15 iterations here with a correct V-cycle, 25 and more with a broken one)."""
    p = I.small_case(dim=3, n=n[0], rho_in=10.0, rho_out=1.0, precision="mixed",
                     poisson_rtol=1e-12, poisson_maxit=200)
    p["n"] = n
    po = O.params_from(p)
    g = O.Grid(3, n, p["L"])
    phi = O.initial_phi(po)
    rhs = I.noise(g.shape, 13) - 0.5
    rhs -= rhs.mean()
    sim = pf.Simulation(p, phi0=phi)
    x, it, relres, st = sim.poisson_solve(rhs)
    assert st == 0 and relres <= 1e-12
    assert it <= 20, it
    res = O.apply_poisson(beta_f32(phi, g, po), x, g) - rhs
    assert np.linalg.norm(res) <= 2e-12 * np.linalg.norm(rhs)
    sim.close()


def test_poisson_mixed_3d_two_sweeps_per_level(pf):
    """V(2,2): the out-of-place sweeps alternate their two buffers; the solve
    converges in fewer inner iterations than with V(1,1)."""
    n = (48, 40, 24)
    p = I.small_case(dim=3, n=n[0], rho_in=10.0, rho_out=1.0, precision="mixed",
                     poisson_rtol=1e-12, poisson_maxit=200)
    p["n"] = n
    p["mg_pre"] = p["mg_post"] = 2
    po = O.params_from(p)
    g = O.Grid(3, n, p["L"])
    phi = O.initial_phi(po)
    rhs = I.noise(g.shape, 13) - 0.5
    rhs -= rhs.mean()
    sim = pf.Simulation(p, phi0=phi)
    x, it, relres, st = sim.poisson_solve(rhs)
    sim.close()
    assert st == 0 and relres <= 1e-12
    assert it <= 12, it
    res = O.apply_poisson(beta_f32(phi, g, po), x, g) - rhs
    assert np.linalg.norm(res) <= 2e-12 * np.linalg.norm(rhs)


def test_unbounded_phi_is_reported(pf):
    """bound_tol > 0: a phase field outside [-bound_tol, 1 + bound_tol] (one cell
    at 1.2, prepared on the host) is reported as PF_ERR_UNBOUNDED, and the same
    field passes when the check is off."""
    p = I.small_case(dim=2, n=32, bound_tol=1e-3)
    po = O.params_from(p)
    phi = O.initial_phi(po)
    phi[7, 9] = 1.2
    sim = pf.Simulation(p, phi0=phi)
    with pytest.raises(pf.PFError) as e:
        sim.diagnostics()
    assert e.value.status == pf.B.PF_ERR_UNBOUNDED
    sim.close()
    sim = pf.Simulation(dict(p, bound_tol=0.0), phi0=phi)
    assert sim.diagnostics()["phi_max"] == pytest.approx(1.2)
    sim.close()


@pytest.mark.parametrize("dim,n,precision,tol", [(2, 32, "fp64", 1e-12), (3, 32, "mixed", 1e-5)])
def test_rk4_shear_mode_amplification_gpu(pf, dim, n, precision, tol):
    """One GPU step of the divergence-free shear mode u_x = A sin(2 pi k y)
    (sigma = 0, uniform fluid) multiplies it by the RK4 stability polynomial
    R(z), z = -nu dt (4/h^2) sin^2(pi k h): the tableau pinned without the
    oracle (the 3D mixed case runs the column-marching stage kernel)."""
    import math

    k, nu, amp = 2, 0.05, 0.3
    p = I.small_case(dim=dim, n=n, sigma=0.0, rho_in=1.0, rho_out=1.0, mu_in=nu, mu_out=nu,
                     pert_mode=0, pert_amp=0.0, precision=precision)
    g = O.Grid(dim, p["n"], p["L"])
    lam = 4.0 / g.h ** 2 * math.sin(math.pi * k * g.h) ** 2
    p["dt"] = 0.5 / (nu * lam)
    z = -0.5
    y = g.centres()[1]
    u0 = amp * np.sin(2.0 * math.pi * k * y)
    sim = pf.Simulation(p, phi0=np.zeros(g.shape))
    sim.set_field("u", u0)
    u0 = sim.field("u")          # as stored (float32 in the mixed path)
    sim.step(1)
    R = 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0
    assert np.max(np.abs(sim.field("u") - R * u0)) <= tol * amp
    assert np.max(np.abs(sim.field("v"))) <= tol * amp
    sim.close()


@pytest.mark.parametrize("n", [(128, 32, 16), (96, 48, 32), (64, 64, 64), (40, 24, 16)])
def test_tma_staged_sweep_matches_cp_async_sweep(pf, n):
    """The finest-level sweep staged by the TMA (tensor boxes for tiles away from
    the periodic seams, cp.async chunks tracked by the mbarriers across them)
    computes exactly what the cp.async-staged sweep computes: with the same 32 x 8
    tiles and two cells per thread the same solution bit for bit and the same
    iteration count, and whole mixed steps agree bit for bit. With the other tile
    shapes (one cell per thread in some sweeps, 32 x 16 tiles) every cell's update is the same
    arithmetic but the fused r.z and z.q dot products sum their partials in
    another order, so the solves agree to that rounding (the
    velocities after two steps, a few 1e-6 at most here, to 1e-4 of their
    maximum: about 1e-10 absolute)."""
    p = I.small_case(dim=3, n=n[0], rho_in=10.0, rho_out=1.0, precision="mixed",
                     poisson_rtol=1e-12, poisson_maxit=200)
    p["n"] = n
    po = O.params_from(p)
    g = O.Grid(3, n, p["L"])
    phi = O.initial_phi(po)
    rhs = I.noise(g.shape, 17) - 0.5
    rhs -= rhs.mean()
    out = []
    for knobs in ({"sweep_staging": 1}, {"sweep_staging": 0, "sweep_tile": 1},
                  {"sweep_staging": 0, "sweep_tile": 0}, {"sweep_staging": 0, "sweep_tile": 2},
                  {"sweep_staging": 0, "sweep_tile": 3}, {"sweep_staging": 0, "sweep_tile": 4}):
        sim = pf.Simulation(dict(p, **knobs), phi0=phi)
        x, it, relres, st = sim.poisson_solve(rhs)
        assert st == 0 and relres <= 1e-12
        sim.step(2)
        out.append((x, it, {c: sim.field(c) for c in ("phi", "u", "v", "w", "p")}))
        sim.close()
    ref, tma8 = out[:2]
    np.testing.assert_array_equal(tma8[0], ref[0])
    assert tma8[1] == ref[1]
    for c in ref[2]:
        np.testing.assert_array_equal(tma8[2][c], ref[2][c])
    for tall in out[2:]:
        assert abs(tall[1] - ref[1]) <= 1
        assert rel(tall[0], ref[0]) < 1e-8
        for c in ref[2]:
            assert rel(tall[2][c], ref[2][c]) < (1e-4 if c in "uvw" else 1e-6), c


@pytest.mark.parametrize("model", ["cdi", "acdi"])
@pytest.mark.parametrize("n", [(48, 16, 12), (96, 24, 20)])
def test_fused_stage_rhs_matches_oracle_and_two_kernel_path(pf, model, n):
    """The fused stage kernel (normals, mu and psi in shared memory) against the
    FP64 oracle on float32-rounded inputs (2e-5 of the phase-field scale, 1e-4 of
    the momentum scale), and against the cell-pass + stage kernels it replaces
    (the same arithmetic: 1e-6 of each field's scale); then two whole RK4 steps
    of both paths agree to float32 rounding."""
    p = I.small_case(dim=3, n=n[0], model=model, precision="mixed")
    p["n"] = n
    p = I.finalize(p)
    po = O.params_from(p)
    g = O.Grid(3, n, p["L"])
    phi = O.initial_phi(po) + 0.01 * (I.noise(g.shape, 19) - 0.5)
    u = rand_velocity(g, 23, amp=0.1)
    out = {}
    for sk in (0, 1):
        sim = pf.Simulation(dict(p, stage_kernel=sk), phi0=phi)
        for d in range(3):
            sim.set_field("uvw"[d], u[d])
        out[sk] = sim.eval_rhs(0.2)
        sim.close()
    phi32 = phi.astype(np.float32).astype(np.float64)
    u32 = [c.astype(np.float32).astype(np.float64) for c in u]
    kphi, ku = out[0]
    assert rel(kphi, O.phase_rhs(phi32, u32, g, po, 0.2)) < 2e-5
    want_u = O.momentum_rhs(phi32, u32, g, po)
    for d in range(3):
        assert rel(ku[d], want_u[d]) < 1e-4, d
    assert rel(kphi, out[1][0]) < 1e-6
    for d in range(3):
        assert rel(ku[d], out[1][1][d]) < 1e-6, d
    fields = {}
    for sk in (0, 1):
        sim = pf.Simulation(dict(p, stage_kernel=sk, poisson_rtol=1e-10), phi0=phi32)
        sim.step(2)
        fields[sk] = {c: sim.field(c) for c in ("phi", "u", "v", "w", "p")}
        sim.close()
    for c in fields[0]:
        assert rel(fields[0][c], fields[1][c]) < 1e-5, c
