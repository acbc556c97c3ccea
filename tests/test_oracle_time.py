"""Pins of the oracle's time integrator and kinetic energy against closed forms.

The paper integrates in time with RK4 (Section 3). For a problem whose
semi-discrete form is linear with a known eigenvalue z / dt on the initial
field, one step of the classical RK4 tableau multiplies that field by the
stability polynomial R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 exactly (forward
Euler: 1 + z). Two such problems isolate the two halves of the step:

* momentum: sigma = 0, uniform density and viscosity, the shear mode
  u_x = A sin(2 pi k y). It is divergence free (the projection leaves it
  alone), has no advection, and the discrete viscous operator multiplies it
  by -nu lambda, lambda = (4 / h^2) sin^2(pi k h);
* phase field: Gamma -> 0, uniform velocity U, phi = 1/2 + a sin(2 pi k x).
  The central advective flux gives the mode the eigenvalue -i U sin(theta) / h,
  theta = 2 pi k h.

Both reference values are written from the tableau and the stencil symbols,
not from the oracle's step. A wrong weight, a stage built from the weight
instead of the stage time, or an accumulator off by one stage changes the
polynomial and fails the exact tests; the order tests show the fourth-order
global error of the integrator against exp(z). The kinetic energy pins use
fields whose face sums are known exactly.
"""
import math

import numpy as np
import pytest

import pf_inputs as I
from oracle import pf_oracle as O


def rk4_poly(z):
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0


def shear_case(n=16, k=2, nu=0.05, amp=0.3, dt=None, scheme="rk4", dim=2):
    """Uniform fluid, no surface tension, u_x = amp sin(2 pi k y) on the x-faces."""
    p = I.small_case(dim=dim, n=n, sigma=0.0, rho_in=1.0, rho_out=1.0, mu_in=nu, mu_out=nu,
                     pert_mode=0, pert_amp=0.0, scheme=scheme)
    if dt is not None:
        p["dt"] = dt
    po = O.params_from(p)
    g = O.Grid(dim, p["n"], p["L"])
    y = g.centres()[1]
    u = [np.zeros(g.shape) for _ in range(dim)]
    u[0] = amp * np.sin(2.0 * math.pi * k * y)
    st = O.State(np.zeros(g.shape), u, np.zeros(g.shape))
    lam = 4.0 / g.h ** 2 * math.sin(math.pi * k * g.h) ** 2
    return po, g, st, -nu * lam


def advect_case(n=32, k=3, U=0.7, a=0.1, dt=None, scheme="rk4"):
    """phi = 1/2 + a sin(2 pi k x) carried by a uniform U with Gamma -> 0."""
    p = I.small_case(dim=2, n=n, sigma=0.0, rho_in=1.0, rho_out=1.0, mu_in=0.01, mu_out=0.01,
                     pert_mode=0, pert_amp=0.0, scheme=scheme, gamma_fixed=1e-300)
    if dt is not None:
        p["dt"] = dt
    po = O.params_from(p)
    g = O.Grid(2, p["n"], p["L"])
    x = g.centres()[0]
    phi = 0.5 + a * np.sin(2.0 * math.pi * k * x)
    u = [U * np.ones(g.shape), np.zeros(g.shape)]
    st = O.State(phi, u, np.zeros(g.shape))
    theta = 2.0 * math.pi * k * g.h
    zc = -1j * U * math.sin(theta) / g.h          # eigenvalue of the mode, times dt below
    return po, g, st, x, zc


def advected_phi(x, k, a, amp):
    """1/2 + a Im(amp e^{i 2 pi k x}): the mode multiplied by the complex factor amp."""
    return 0.5 + a * np.imag(amp * np.exp(1j * 2.0 * math.pi * k * x))


# --------------------------------------------------------------------------
# exact one-step amplification
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_rk4_shear_mode_amplification_is_the_rk4_polynomial(dim):
    n = 16 if dim == 2 else 8
    _, _, _, z0 = shear_case(n=n, dim=dim)
    po, g, st, _ = shear_case(n=n, dim=dim, dt=-0.5 / z0)     # z = -0.5
    z = z0 * po["dt"]
    out = O.step(st, po)
    want = rk4_poly(z) * st.u[0]
    assert np.max(np.abs(out.u[0] - want)) <= 1e-14 * np.max(np.abs(st.u[0]))
    for d in range(1, dim):
        assert np.max(np.abs(out.u[d])) <= 1e-15
    assert np.max(np.abs(out.p)) <= 1e-12
    # the check has teeth: z is not small, so R(z) differs from 1 + z, exp(z)
    assert abs(rk4_poly(z) - (1 + z)) > 1e-3 and abs(rk4_poly(z) - math.exp(z)) > 1e-6


def test_forward_euler_shear_mode_amplification():
    po, g, st, z0 = shear_case(dt=0.02, scheme="fe")
    out = O.step(st, po)
    assert np.max(np.abs(out.u[0] - (1.0 + z0 * po["dt"]) * st.u[0])) <= 1e-14


def test_rk4_advected_mode_amplification_is_the_rk4_polynomial():
    po, g, st, x, zc = advect_case(dt=0.05)          # |z| = 0.44
    z = zc * po["dt"]
    out = O.step(st, po)
    want = advected_phi(x, 3, 0.1, rk4_poly(z))
    assert np.max(np.abs(out.phi - want)) <= 2e-15
    # the velocity stays uniform (no force, uniform density: nothing to project)
    assert np.max(np.abs(out.u[0] - 0.7)) <= 1e-15
    assert abs(abs(rk4_poly(z)) - 1.0) > 1e-7   # RK4's slight damping of the rotation is seen


# --------------------------------------------------------------------------
# temporal order (global error against the exact semi-discrete solution)
# --------------------------------------------------------------------------
def _orders(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_rk4_fourth_order_in_time_shear_mode():
    T = 1.0 / -shear_case()[3]      # one e-folding of the mode
    errs = []
    for nsteps in (4, 8, 16):
        po, g, st, z0 = shear_case(dt=T / nsteps)
        for _ in range(nsteps):
            st = O.step(st, po)
        _, _, s0, _ = shear_case(dt=T / nsteps)
        errs.append(np.max(np.abs(st.u[0] - math.exp(z0 * T) * s0.u[0])))
    for o in _orders(errs):
        assert 3.8 < o < 4.2, (errs, _orders(errs))


def test_forward_euler_first_order_in_time_shear_mode():
    T = 1.0 / -shear_case()[3]
    errs = []
    for nsteps in (12, 24, 48):
        po, g, st, z0 = shear_case(dt=T / nsteps, scheme="fe")
        for _ in range(nsteps):
            st = O.step(st, po)
        _, _, s0, _ = shear_case(dt=T / nsteps)
        errs.append(np.max(np.abs(st.u[0] - math.exp(z0 * T) * s0.u[0])))
    for o in _orders(errs):
        assert 0.85 < o < 1.15, (errs, _orders(errs))


def test_rk4_fourth_order_in_time_advected_mode():
    T = 0.3
    errs = []
    for nsteps in (4, 8, 16):
        po, g, st, x, zc = advect_case(dt=T / nsteps)
        for _ in range(nsteps):
            st = O.step(st, po)
        errs.append(np.max(np.abs(st.phi - advected_phi(x, 3, 0.1, np.exp(zc * T)))))
    for o in _orders(errs):
        assert 3.8 < o < 4.2, (errs, _orders(errs))


# --------------------------------------------------------------------------
# the pins have teeth: a plausible mistake planted in the oracle fails them
# --------------------------------------------------------------------------
@pytest.mark.parametrize("attr,bad", [
    ("RK4_W", (0.25, 0.25, 0.25, 0.25)),            # equal weights
    ("RK4_W", (1.0 / 6.0, 1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0)),  # weights shifted by a stage
    ("RK4_C", (0.0, 1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0)),  # stages built from the weights
    ("RK4_C", (0.0, 0.5, 1.0, 1.0)),                 # a wrong stage time
])
def test_planted_tableau_mistakes_fail_the_amplification_pin(monkeypatch, attr, bad):
    po, g, st, z0 = shear_case(dt=0.02)
    monkeypatch.setattr(O, attr, bad)
    out = O.step(st, po)
    err = np.max(np.abs(out.u[0] - rk4_poly(z0 * po["dt"]) * st.u[0]))
    assert err > 1e-7 * np.max(np.abs(st.u[0]))


# --------------------------------------------------------------------------
# kinetic energy, KE = 1/2 sum_faces rho_f u_d^2 dV
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_kinetic_energy_uniform_flow(dim):
    p = I.small_case(dim=dim, n=16 if dim == 2 else 8, rho_in=3.0, rho_out=3.0)
    po = O.params_from(p)
    g = O.Grid(dim, p["n"], p["L"])
    vel = (0.4, -0.7, 0.2)[:dim]
    st = O.State(np.full(g.shape, 0.3), [c * np.ones(g.shape) for c in vel], np.zeros(g.shape))
    ke = O.diagnostics(st, po)["ke"]
    assert abs(ke - 0.5 * 3.0 * sum(c * c for c in vel) * p["L"] ** dim) <= 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_kinetic_energy_two_density_slab(dim):
    """phi = 1 on the lower half (rows j < ny/2), 0 above: every x- (and z-) face
    lies inside one phase and the y-faces average across the two interfaces, so
    sum_faces rho_f dV = (rho_in + rho_out) |box| / 2 for each component and
    KE = (rho_in + rho_out) |U|^2 |box| / 4."""
    n = 16 if dim == 2 else 8
    p = I.small_case(dim=dim, n=n, rho_in=7.0, rho_out=0.5)
    po = O.params_from(p)
    g = O.Grid(dim, p["n"], p["L"])
    y = g.centres()[1]
    phi = (y < 0.5 * p["L"]).astype(np.float64)
    vel = (0.4, -0.7, 0.2)[:dim]
    st = O.State(phi, [c * np.ones(g.shape) for c in vel], np.zeros(g.shape))
    ke = O.diagnostics(st, po)["ke"]
    want = 0.25 * (7.0 + 0.5) * sum(c * c for c in vel) * p["L"] ** dim
    assert abs(ke - want) <= 1e-14 * want


def test_kinetic_energy_shear_mode():
    """u_x = A sin(2 pi k y): the sum of sin^2 over whole periods is n/2, so
    KE = rho A^2 |box| / 4."""
    po, g, st, _ = shear_case(n=16, amp=0.3)
    ke = O.diagnostics(st, dict(po, sigma=1.0))["ke"]    # Ca_inf divides by sigma
    assert abs(ke - 0.25 * 1.0 * 0.09) <= 1e-15
