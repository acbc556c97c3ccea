"""Pins of the oracle's ACDI phase field (the accurate conservative diffuse-interface
model of Jain, J. Comput. Phys. 469, 2022, which the 256^2 and 384^3 workloads
name; this paper does not define it).

The model is the CDI flux form with the sharpening term phi (1 - phi) n
replaced by (1/4) [1 - tanh^2(psi_f / (2 eps))] n_f, psi = eps ln(phi / (1 - phi))
the signed-distance-like variable and n the normals of psi. What fixes it
independently of the oracle:

* psi of the equilibrium tanh profile is the signed distance itself;
* the sharpening coefficient equals phi (1 - phi) of the same cell's phi
  (an algebraic identity), and at a face of a flat equilibrium profile it
  equals phi (1 - phi) of the analytic profile at the face (where CDI's
  two-cell mean of phi is off by O(h^2));
* the flat tanh profile is steady up to the O(h^2) error of the diffusive
  face difference, and that error converges at second order;
* the fluxes telescope (sum of the right-hand side is zero) and forward
  Euler keeps 0 <= phi <= 1 at eps = dx, Gamma = max |u|;
* without sharpening and diffusion (Gamma -> 0) the right-hand side is CDI's.
"""
import math

import numpy as np
import pytest

import pf_inputs as I
from oracle import pf_oracle as O


def params(dim=2, n=32, **kw):
    base = dict(model="acdi", pert_mode=0, pert_amp=0.0)
    base.update(kw)
    return O.params_from(I.small_case(dim=dim, n=n, **base))


def flat_profile(g, eps, x0=0.5, d=0):
    """phi = [1 + tanh((x0 - x)/(2 eps))] / 2 along axis d, and the signed distance."""
    x = g.centres()[d]
    s = x0 - x
    return 0.5 * (1.0 + np.tanh(s / (2.0 * eps))), s


def test_psi_is_the_signed_distance_of_the_equilibrium_profile():
    g = O.Grid(2, (64, 64))
    eps = 1.0 / 64
    phi, s = flat_profile(g, eps)
    psi = O.acdi_psi(phi, eps)
    band = np.abs(s) < 10 * eps
    assert np.max(np.abs(psi[band] - s[band])) < 1e-6 * eps
    # saturated cells stay finite: |psi| <= eps ln(1 / eps0)
    assert np.all(np.isfinite(psi)) and np.max(np.abs(psi)) <= eps * math.log(1e20) * (1 + 1e-12)


def test_sharpening_coefficient_identity_at_cells():
    g = O.Grid(2, (32, 32))
    eps = 1.0 / 32
    phi = 0.02 + 0.96 * I.noise(g.shape, 3)
    psi = O.acdi_psi(phi, eps)
    assert np.max(np.abs(O.acdi_sharpening(psi, eps) - phi * (1.0 - phi))) < 1e-13


@pytest.mark.parametrize("n", [32, 64])
def test_face_sharpening_is_the_profile_value_at_the_face(n):
    """Flat profile along x: psi is linear, so its face mean is the face's signed
    distance and the coefficient is phi(1 - phi) of the analytic profile there
    (to rounding); CDI's two-cell phi mean differs at O(h^2)."""
    g = O.Grid(2, (n, n))
    eps = 1.0 / n
    phi, s = flat_profile(g, eps)
    psi = O.acdi_psi(phi, eps)
    sf = O.face_avg(s, g, 0)                         # signed distance of the x-faces
    pf_exact = 0.5 * (1.0 + np.tanh(sf / (2.0 * eps)))
    want = pf_exact * (1.0 - pf_exact)
    got = O.acdi_sharpening(O.face_avg(psi, g, 0), eps)
    inner = np.abs(sf) < 0.25                        # away from the periodic seam's kink
    assert np.max(np.abs(got - want)[inner]) < 1e-9
    pf = O.face_avg(phi, g, 0)
    assert np.max(np.abs(pf * (1 - pf) - want)[inner]) > 1e-3


def test_flat_profile_steady_to_second_order():
    """Gamma = 1, u = 0: the right-hand side on the flat tanh profile (eps = 1/16
    fixed, h refined) falls at second order in h (the face difference's
    truncation error)."""
    errs = []
    for n in (32, 64, 128):
        p = params(dim=2, n=n, eps=1.0 / 16)
        g = O.Grid(2, p["n"], p["L"])
        phi, s = flat_profile(g, p["eps"])
        u = [np.zeros(g.shape), np.zeros(g.shape)]
        r = O.phase_rhs(phi, u, g, p, 1.0)
        inner = np.abs(s) < 0.25
        errs.append(float(np.max(np.abs(r[inner]))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < o < 2.3 for o in orders), (errs, orders)


def test_fluxes_telescope_and_forward_euler_bounded():
    """Sum of the right-hand side vanishes (telescoping fluxes); forward Euler in
    a divergence-free random velocity with Gamma = max |u| and eps = dx keeps
    0 <= phi <= 1 and the mass."""
    p = params(dim=2, n=32)
    g = O.Grid(2, p["n"], p["L"])
    rng = np.random.default_rng(6)
    # divergence-free face velocity from a random streamfunction at cell corners
    sf = rng.standard_normal(g.shape)
    u = [(np.roll(sf, -1, axis=0) - sf) / g.h, -(np.roll(sf, -1, axis=1) - sf) / g.h]
    assert np.max(np.abs(O.divergence(u, g))) < 1e-9
    phi = O.initial_phi(dict(p, pert_mode=2, pert_amp=0.1))
    gam = max(np.max(np.abs(c)) for c in u)
    dt = 0.1 * g.h / (gam * 4)
    m0 = phi.sum()
    for _ in range(100):
        rhs = O.phase_rhs(phi, u, g, p, gam)
        assert abs(rhs.sum()) < 1e-8 * np.max(np.abs(rhs)) * rhs.size
        phi = phi + dt * rhs
    assert abs(phi.sum() - m0) < 1e-12 * m0
    assert phi.min() >= 0.0 and phi.max() <= 1.0


def test_pure_advection_equals_cdi():
    p = params(dim=3, n=12)
    g = O.Grid(3, p["n"], p["L"])
    phi = O.initial_phi(dict(p, pert_mode=2, pert_amp=0.1))
    u = [0.3 * (I.noise(g.shape, 5 + d) - 0.5) for d in range(3)]
    a = O.phase_rhs(phi, u, g, p, 0.0)
    b = O.phase_rhs(phi, u, g, dict(p, model=O.MODEL_CDI), 0.0)
    np.testing.assert_array_equal(a, b)
    # with sharpening the two models differ at O(h^2) of the interface band
    c = O.phase_rhs(phi, u, g, p, 0.5)
    d = O.phase_rhs(phi, u, g, dict(p, model=O.MODEL_CDI), 0.5)
    assert 0 < np.max(np.abs(c - d)) < 0.2 * np.max(np.abs(d))
