"""The exact standing-wave amplitude used by the Section 3.2 study
(Prosperetti 1981), checked against what fixes it independently: it starts at
a(0) = 1 from rest, reduces to the inviscid linear wave cos(w0 t) with
w0^2 = sigma k^3 / (rho1 + rho2) as nu -> 0 (with an O(sqrt(nu)) correction),
and decays at the rate of the interfacial Stokes layer."""
import math

import numpy as np

from paper_2205_05835_gb300.studies import prosperetti_amplitude, wave_eps


def test_starts_at_one_from_rest():
    t = np.array([0.0, 1e-6, 2e-6])
    a = prosperetti_amplitude(t, 1.0, 0.064720863, 2.0, 1.0, 1.0)
    assert abs(a[0] - 1.0) < 1e-12
    assert abs(a[2] - a[0]) < 1e-6       # no initial velocity: flat start


def test_inviscid_limit_is_linear_capillary_wave():
    t = np.linspace(0.0, 20.0, 2001)
    for sigma, k, r1, r2 in ((2.0, 1.0, 1.0, 1.0), (1.0, 2.0, 1.0, 3.0)):
        w0 = math.sqrt(sigma * k ** 3 / (r1 + r2))
        err = [np.max(np.abs(prosperetti_amplitude(t, k, nu, sigma, r1, r2) - np.cos(w0 * t)))
               for nu in (1e-6, 1e-8)]
        # the correction scales like sqrt(nu): a hundred times smaller nu, ten times smaller error
        assert err[0] < 0.02 and err[1] < 0.11 * err[0] + 1e-9, err


def test_interfacial_boundary_layer_damping():
    """Between two viscous fluids the tangential velocity of the inviscid wave
    jumps across the interface; the Stokes layer that smooths the jump damps
    the wave at a rate proportional to sqrt(nu omega0) k (not nu k^2 as for a
    free surface). For equal densities the rate is k sqrt(nu omega0) / (2
    sqrt 2): the peaks of the exact solution decay accordingly, and ten times
    the viscosity gives sqrt(10) times the rate."""
    k, w0 = 1.0, 1.0
    rates = []
    for nu in (1e-3, 1e-4):
        t = np.linspace(0.0, 40.0, 400001)
        a = prosperetti_amplitude(t, k, nu, 2.0, 1.0, 1.0)
        tm = [2 * math.pi * m / w0 for m in (3, 5)]
        pk = [float(a[np.abs(t - x) < 0.5].max()) for x in tm]
        rate = math.log(pk[0] / pk[1]) / (tm[1] - tm[0])
        rates.append(rate)
        want = k * math.sqrt(nu * w0) / (2.0 * math.sqrt(2.0))
        assert abs(rate / want - 1.0) < 0.05, (nu, rate, want)
    assert abs(rates[0] / rates[1] / math.sqrt(10.0) - 1.0) < 0.05


def test_wave_eps_panels():
    L = 2 * math.pi
    assert wave_eps("h", 64) == L / 32
    # dx = 32^(1/2) eps^(3/2) in units of the box edge
    for n in (16, 64, 256):
        e = wave_eps("eps", n) / L
        assert abs(math.sqrt(32.0) * e ** 1.5 - 1.0 / n) < 1e-12
