"""Seeded, synthetic inputs shared by the oracle, the tests and bench.py.

This module holds workload tables and random-number generators only. It
contains none of the discrete method's arithmetic: no stencil, no phase-field
or momentum right-hand side, no pressure solve, no initial profile. Both the
CUDA path's tests and the FP64 oracle take their parameters from here so that
they run the identical problem.

Workloads follow the paper's canonical static-drop test (Section 3.1: a drop
of radius R in a unit box, sigma = 1, Laplace number La = sigma*rho*D/mu^2)
and a mode-n oscillating drop, on periodic unit boxes.
"""
from __future__ import annotations

import copy
import json
import math

import numpy as np

# Enumerations shared with the C ABI (same integer values as include/pf.h).
MODELS = {"cdi": 0, "sb": 1, "isodi": 2, "acdi": 3}
FORCES = {"eb": 0, "csf": 1, "lcsf": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
SCHEMES = {"rk4": 0, "fe": 1}
MOMENTUM = {"advective": 0, "consistent": 1}
SHAPES = {"drop": 0, "wave": 1}

BATCH_SEED = 20261203


def _base(**kw):
    p = dict(
        dim=2, n=(64, 64, 1), L=1.0,
        model="cdi", force="eb", precision="fp64", scheme="rk4",
        sigma=1.0, eps=None, rho_in=1.0, rho_out=1.0, mu_in=0.1, mu_out=0.1,
        gamma_fixed=0.0, gamma_min=0.0, dt=None, delta_n=1e-12, momentum="advective",
        wall_y=0, shape="drop",
        poisson_rtol=1e-12, poisson_maxit=200,
        R=0.25, pert_mode=0, pert_amp=0.0, steps=1,
    )
    p.update(kw)
    return p


def finalize(p):
    """Fill derived defaults: eps = dx and dt from stability limits."""
    p = copy.deepcopy(p)
    n = tuple(int(v) for v in p["n"])
    if p["dim"] == 2:
        n = (n[0], n[1], 1)
    p["n"] = n
    dx = p["L"] / n[0]
    if p["eps"] is None:
        p["eps"] = dx
    if p["dt"] is None:
        p["dt"] = suggest_dt(p)
    return p


def suggest_dt(p):
    """Half the smallest of the capillary, viscous and advective limits.

    Capillary: sqrt((rho_in + rho_out) dx^3 / (4 pi sigma)) (Brackbill-type
    limit); viscous: dx^2 / (2 d nu_max). The phase-field limit
    dx^2/(2 d gamma eps) is applied when gamma is fixed.
    """
    dx = p["L"] / p["n"][0]
    d = p["dim"]
    lims = [0.2 * dx]   # without surface tension: an advective bound for velocities of order 1
    if p["sigma"] > 0:
        lims = [math.sqrt((p["rho_in"] + p["rho_out"]) * dx ** 3 / (4.0 * math.pi * p["sigma"]))]
    nu = max(p["mu_in"] / p["rho_in"], p["mu_out"] / p["rho_out"])
    if nu > 0:
        lims.append(dx * dx / (2.0 * d * nu))
    if p["gamma_fixed"] > 0:
        eps = p["eps"] if p["eps"] is not None else dx
        lims.append(dx * dx / (2.0 * d * p["gamma_fixed"] * eps))
    return 0.5 * min(lims)


def static_drop_64():
    """64^2 static drop, FP64, CDI + EB, density and viscosity ratio 1, La = 12000.

    La = sigma rho D / mu^2 with sigma = 1, mu = 0.1, D = 0.5 gives rho = 240.
    """
    return finalize(_base(dim=2, n=(64, 64, 1), rho_in=240.0, rho_out=240.0,
                          mu_in=0.1, mu_out=0.1, steps=200))


def static_drop_256_r1000(force="eb", precision="fp64", model="acdi"):
    """256^2 static drop, density ratio 1000, viscosity ratio 100, ACDI phase field."""
    return finalize(_base(dim=2, n=(256, 256, 1), rho_in=240.0, rho_out=0.24,
                          mu_in=0.1, mu_out=0.001, force=force, precision=precision,
                          model=model, steps=2000))


def oscillating_drop_384(precision="mixed", n=384, steps=500, model="acdi"):
    """384^3 mode-2 oscillating drop, amplitude 0.05 R, density/viscosity ratio 10,
    ACDI phase field, energy-based force."""
    return finalize(_base(dim=3, n=(n, n, n), rho_in=10.0, rho_out=1.0,
                          mu_in=0.01, mu_out=0.001, pert_mode=2, pert_amp=0.05,
                          precision=precision, model=model, poisson_rtol=1e-10, steps=steps))


def oscillating_drop_2d_256():
    """256^2 mode-2 oscillating drop used for differentiation, density ratio 10."""
    return finalize(_base(dim=2, n=(256, 256, 1), rho_in=10.0, rho_out=1.0,
                          mu_in=0.01, mu_out=0.001, pert_mode=2, pert_amp=0.05,
                          steps=500))


def batch_manifest(count=256, seed=BATCH_SEED, precision="mixed", poisson_rtol=1e-10):
    """Seeded manifest of 2D drops of uneven sizes and Laplace numbers.

    N ~ U{64, 80, ..., 512}, R ~ U[0.15, 0.3], log10 La ~ U[2, 5],
    density ratio in {1, 10, 1000}, static or mode-2 oscillating 50/50.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.arange(64, 513, 16)
    out = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        R = float(rng.uniform(0.15, 0.3))
        la = float(10.0 ** rng.uniform(2.0, 5.0))
        ratio = float(rng.choice([1.0, 10.0, 1000.0]))
        osc = bool(rng.integers(0, 2))
        sigma, rho_in = 1.0, 1.0
        mu = math.sqrt(sigma * rho_in * 2.0 * R / la)
        out.append(finalize(_base(dim=2, n=(n, n, 1), R=R, rho_in=rho_in,
                                  rho_out=rho_in / ratio, mu_in=mu, mu_out=mu,
                                  pert_mode=2 if osc else 0,
                                  pert_amp=0.05 if osc else 0.0, steps=1000,
                                  precision=precision, poisson_rtol=poisson_rtol)))
    return out


def standing_wave(n=64, force="eb", model="cdi", precision="fp64", eps_frac=1.0 / 32,
                  steps=1000, **kw):
    """Section 3.2 standing wave on an n x n grid: a 2 pi x 2 pi box, periodic in
    x, free-slip walls at y = 0 and y = 2 pi; interface y = pi - A0 cos(x - dx/2)
    with A0 = 2 pi / 100 (one wavelength across the box), sigma = 2,
    rho = 1 and nu = 0.064720863 in both phases, dt = 0.003 unless the
    stability bound of suggest_dt is smaller. eps = eps_frac * 2 pi: the
    paper's eps = 1/32 is read in units of the box edge (it quotes
    eps / dx = 2 on the 64 x 64 mesh)."""
    L = 2.0 * math.pi
    nu = 0.064720863
    p = _base(dim=2, n=(n, n, 1), L=L, model=model, force=force, precision=precision,
              sigma=2.0, rho_in=1.0, rho_out=1.0, mu_in=nu, mu_out=nu, eps=eps_frac * L,
              R=math.pi, pert_mode=1, pert_amp=0.02, shape="wave", wall_y=1, steps=steps,
              poisson_rtol=1e-12 if precision == "fp64" else 1e-10)
    p.update(kw)
    if p["dt"] is None:
        p["dt"] = min(0.003, suggest_dt(p))
    return finalize(p)


def small_case(dim=2, n=32, **kw):
    """Small periodic drop for parity tests; any keyword overrides a parameter."""
    base = dict(dim=dim, n=(n, n, n if dim == 3 else 1), rho_in=10.0, rho_out=1.0,
                mu_in=0.01, mu_out=0.005, pert_mode=2, pert_amp=0.05, R=0.25)
    base.update(kw)
    return finalize(_base(**base))


def noise(shape, seed, lo=0.0, hi=1.0):
    """Seeded uniform noise (PCG64) for stencil tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)


def to_json(p):
    return json.dumps({k: (list(v) if isinstance(v, tuple) else v) for k, v in p.items()},
                      sort_keys=True)
