"""Pins of the oracle's free-slip walls in y (Section 3.2 standing wave).

The walled oracle evaluates every stencil on image rows beyond the walls and
solves a pressure equation with zero face coefficients on the wall faces. It
is pinned against the periodic oracle (itself pinned in test_oracle_pins.py)
through the method of images: a mirror-symmetric state on the box doubled in
y is a periodic state whose lower half evolves exactly like the walled box,
because every stencil is symmetric under the reflection. So the walled
right-hand sides, projection and whole steps must equal the lower half of the
periodic ones on the doubled box; a wrong image parity, a dropped wall
condition or a wall face shifted by one fails these. Conservation, zero
normal velocity and the wave's initial profile are checked directly.
"""
import math

import numpy as np
import pytest

import pf_inputs as I
from oracle import pf_oracle as O


def walled_case(n=(16, 12), model="cdi", force="eb", **kw):
    base = dict(dim=2, n=(n[0], n[1], 1), L=1.0, model=model, force=force, wall_y=1,
                shape="wave", R=0.5 * n[1] / n[0], pert_mode=1, pert_amp=0.15,
                rho_in=3.0, rho_out=1.0, mu_in=0.02, mu_out=0.01, gamma_fixed=0.3,
                poisson_rtol=1e-12)
    base.update(kw)
    return O.params_from(I.finalize(I._base(**base)))


def doubled(p):
    """The periodic box of twice the height."""
    q = dict(p)
    q["n"] = (p["n"][0], 2 * p["n"][1], 1)
    q["wall_y"] = 0
    return q


def mirror_up(a, odd_face=False):
    """Extend (ny, nx) rows to (2 ny, nx): cells mirror about y = ny h; a
    y-face field is odd about the wall faces (face ny = 0, face ny + j = -face ny - j)."""
    if not odd_face:
        return np.concatenate([a, a[::-1]], axis=0)
    assert np.all(a[0] == 0.0)
    top = np.concatenate([np.zeros_like(a[:1]), -a[:0:-1]], axis=0)
    return np.concatenate([a, top], axis=0)


def state(p, seed):
    """A smooth wave profile with noise, and a random velocity with v = 0 on the walls."""
    g = O.Grid(2, p["n"], p["L"])
    phi = O.initial_phi(p) + 0.03 * (I.noise(g.shape, seed) - 0.5)
    u = 0.2 * (I.noise(g.shape, seed + 1) - 0.5)
    v = 0.2 * (I.noise(g.shape, seed + 2) - 0.5)
    v[0, :] = 0.0
    return g, phi, [u, v]


@pytest.mark.parametrize("model,force", [("cdi", "eb"), ("cdi", "csf"), ("cdi", "lcsf"),
                                         ("sb", "eb"), ("isodi", "lcsf")])
def test_walled_rhs_equals_doubled_periodic(model, force):
    p = walled_case(model=model, force=force)
    q = doubled(p)
    g, phi, u = state(p, 5)
    g2 = O.Grid(2, q["n"], q["L"])
    phi2 = mirror_up(phi)
    u2 = [mirror_up(u[0]), mirror_up(u[1], odd_face=True)]
    ny = p["n"][1]
    gam = 0.3
    kw = O.phase_rhs_walls(phi, u, g, p, gam)
    kp = O.phase_rhs(phi2, u2, g2, q, gam)
    np.testing.assert_allclose(kw, kp[:ny], rtol=0, atol=1e-12 * np.abs(kp).max())
    mw = O.momentum_rhs_walls(phi, u, g, p)
    mp = O.momentum_rhs(phi2, u2, g2, q)
    for d in range(2):
        np.testing.assert_allclose(mw[d], mp[d][:ny], rtol=0, atol=1e-12 * np.abs(mp[d]).max())
    # the periodic right-hand side of the wall's normal velocity vanishes by
    # symmetry; the walled one is zero by the wall condition
    assert np.abs(mp[1][0]).max() < 1e-12 * np.abs(mp[1]).max()
    assert np.all(mw[1][0] == 0.0)


def test_walled_projection_equals_doubled_periodic():
    p = walled_case()
    q = doubled(p)
    g, phi, u = state(p, 9)
    g2 = O.Grid(2, q["n"], q["L"])
    tau = 1e-3
    uw, pw = O.project(u, phi, g, p, tau)
    up, pp = O.project([mirror_up(u[0]), mirror_up(u[1], True)], mirror_up(phi), g2, q, tau)
    ny = p["n"][1]
    np.testing.assert_allclose(pw, pp[:ny], rtol=0, atol=1e-10 * np.abs(pp).max())
    for d in range(2):
        np.testing.assert_allclose(uw[d], up[d][:ny], rtol=0, atol=1e-10 * np.abs(up[d]).max())
    # divergence free in every cell, the walls' normal velocity untouched (zero)
    assert np.abs(O.divergence(uw, g)).max() < 1e-9 * np.abs(u[0]).max() / g.h
    assert np.all(uw[1][0] == 0.0)


@pytest.mark.parametrize("scheme", ["rk4", "fe"])
def test_walled_step_equals_doubled_periodic(scheme):
    p = walled_case(scheme=scheme, force="lcsf")
    q = doubled(p)
    g, phi, u = state(p, 13)
    u = [0.1 * c for c in u]
    st = O.step(O.State(phi, u, np.zeros(g.shape)), p)
    st2 = O.step(O.State(mirror_up(phi), [mirror_up(u[0]), mirror_up(u[1], True)],
                         np.zeros((2 * p["n"][1], p["n"][0]))), q)
    ny = p["n"][1]
    np.testing.assert_allclose(st.phi, st2.phi[:ny], rtol=0, atol=1e-12)
    for d in range(2):
        np.testing.assert_allclose(st.u[d], st2.u[d][:ny], rtol=0,
                                   atol=1e-10 * np.abs(st2.u[d]).max())
    np.testing.assert_allclose(st.p, st2.p[:ny], rtol=0, atol=1e-10 * np.abs(st2.p).max())


def test_walled_surface_energy_equals_half_doubled():
    p = walled_case()
    g, phi, _ = state(p, 3)
    q = doubled(p)
    g2 = O.Grid(2, q["n"], q["L"])
    se_w = O.surface_energy(phi, g, p["sigma"], p["eps"], wall_y=1)
    se_p = O.surface_energy(mirror_up(phi), g2, p["sigma"], p["eps"])
    assert abs(se_w - 0.5 * se_p) < 1e-12 * se_p


def test_standing_wave_profile():
    """The wave's interface y0 - A0 cos(k (x - dx/2)): the column integral of phi
    at x = dx/2 recovers y0 - A0, up to the tanh tails cut by the walls eight
    widths 2 eps away (about eps exp(-16) = 2e-8)."""
    p = O.params_from(I.standing_wave(n=64))
    assert p["eps"] == pytest.approx(2 * math.pi / 32) and p["dt"] == 0.003
    g = O.Grid(2, p["n"], p["L"])
    phi = O.initial_phi(p)
    A0 = 2 * math.pi / 100
    col = float(np.sum(phi[:, 0])) * g.h
    assert abs((p["R"] - col) - A0 * math.cos(0.0)) < 1e-7
    # a quarter wavelength on: cos(pi/2) = 0, the mean height
    col_q = float(np.sum(phi[:, 16])) * g.h
    assert abs(col_q - p["R"]) < 1e-7


def test_walled_wave_conserves_mass_and_keeps_walls_closed():
    p = O.params_from(I.standing_wave(n=32))
    st = O.initial_state(p)
    m0 = float(np.sum(st.phi))
    g = O.Grid(2, p["n"], p["L"])
    for _ in range(20):
        st = O.step(st, p)
    assert abs(float(np.sum(st.phi)) / m0 - 1.0) < 1e-13
    assert np.all(st.u[1][0] == 0.0)
    assert np.abs(O.divergence(st.u, g)).max() < 1e-10
    # the wave moves: the interface at x = dx/2 has started down
    A = p["R"] - float(np.sum(st.phi[:, 0])) * g.h
    assert A < 2 * math.pi / 100
