"""FP64 CPU oracle for one fractional time step of the one-fluid, variable-density,
incompressible two-phase solver with a second-order phase field and the
energy-based surface tension force (Mirjalili, Khanwale & Mani, "Assessment of
an energy-based surface tension model for simulation of two-phase flows using
second-order phase field methods", arXiv 2205.05835).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import or call this module; the CUDA product
path never does, and the two share no code. Everything here is plain numpy in
float64: every stencil is a whole-array expression built from periodic shifts
(np.roll) in the order the formulas are written, with no blocking or fusion.
The pressure Poisson equation is solved exactly by a sparse direct solver
(scipy SuperLU), which is the plain definition of the projection.

Discretization (the paper defers it to its reference [Mirjalili 2021]; the
readings below are this implementation's):
  * uniform periodic Cartesian grid, dx = dy (= dz) = L / n, cell centres at
    (i + 1/2) dx; arrays are shaped (ny, nx) in 2D and (nz, ny, nx) in 3D so
    x is the fastest index;
  * phi, the chemical potential, curvature and pressure live at cell centres;
    velocity component d lives on the d-faces, and face i - 1/2 is stored at
    index i (between cells i - 1 and i);
  * central second-order differences everywhere; projected RK4 or forward
    Euler in time;
  * optionally free-slip walls at y = 0 and y = ny h instead of periodicity in
    y (the standing wave of Section 3.2), imposed through image rows.

Parity status: every function below is pinned by tests/test_oracle_pins.py
against closed forms, invariants, brute-force matrices or exact solutions,
except where a function's docstring says "parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import eval_legendre

MODEL_CDI, MODEL_SB, MODEL_ISODI, MODEL_ACDI = 0, 1, 2, 3
FORCE_EB, FORCE_CSF, FORCE_LCSF = 0, 1, 2
SCHEME_RK4, SCHEME_FE = 0, 1
MOMENTUM_ADVECTIVE, MOMENTUM_CONSISTENT = 0, 1

_MODELS = {"cdi": 0, "sb": 1, "isodi": 2, "acdi": 3}
_FORCES = {"eb": 0, "csf": 1, "lcsf": 2}
_SCHEMES = {"rk4": 0, "fe": 1}
_MOMENTUM = {"advective": 0, "consistent": 1}
_SHAPES = {"drop": 0, "wave": 1}
SHAPE_DROP, SHAPE_WAVE = 0, 1

# Projected RK4 (classical tableau): stage time fractions and weights.
RK4_C = (0.0, 0.5, 0.5, 1.0)
RK4_W = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


# ----------------------------------------------------------------------------
# grid helpers
# ----------------------------------------------------------------------------
class Grid:
    """Periodic uniform grid; shape is (ny, nx) in 2D or (nz, ny, nx) in 3D."""

    def __init__(self, dim, n, L=1.0):
        self.dim = int(dim)
        n = tuple(int(v) for v in n)
        self.n = n[: self.dim]                      # (nx, ny[, nz])
        self.shape = tuple(reversed(self.n))        # numpy shape, x fastest
        self.L = float(L)
        self.h = self.L / self.n[0]
        self.dV = self.h ** self.dim

    def axis(self, d):
        return self.dim - 1 - d

    def centres(self):
        """Cell-centre coordinates (x, y[, z]) as broadcast arrays."""
        coords = []
        for d in range(self.dim):
            c = (np.arange(self.n[d]) + 0.5) * self.h
            shp = [1] * self.dim
            shp[self.axis(d)] = self.n[d]
            coords.append(c.reshape(shp) * np.ones(self.shape))
        return coords


def S(a, g, d, k):
    """Periodic shift: S(a, d, k)[i] = a[i + k e_d]."""
    return np.roll(a, -k, axis=g.axis(d))


def params_from(p):
    """Normalise a parameter dict (names from pf_inputs) to oracle form."""
    q = dict(p)
    for key, table in (("model", _MODELS), ("force", _FORCES), ("scheme", _SCHEMES),
                       ("momentum", _MOMENTUM), ("shape", _SHAPES)):
        if isinstance(q.get(key), str):
            q[key] = table[q[key]]
    return q


# ----------------------------------------------------------------------------
# initial condition (Section 2, footnote to the definition of sigma-hat)
# ----------------------------------------------------------------------------
def initial_phi(p):
    """phi0 = [1 + tanh(s / (2 eps))] / 2 with s the signed distance, phi = 1 in
    the drop (Section 2, footnote on the equilibrium profile).

    The drop is centred in the box (at n_d h / 2 along each axis). Its radius is R(theta) = R (1 + a cos(n
    theta)) in 2D and R (1 + a P_n(cos theta)) in 3D (theta measured from the z
    axis); R(theta) - r is taken as the signed distance for a perturbed drop.

    Standing wave (shape 1, Section 3.2, 2D): the interface height is
    y0 - A0 cos(k (x - dx/2)) with y0 = R and A0 = a R, k = 2 pi n / (nx h) (n
    wavelengths across the box); y_i(x) - y is the signed distance, phi = 1
    below the interface.
    """
    g = Grid(p["dim"], p["n"], p["L"])
    X = g.centres()
    if p.get("shape", SHAPE_DROP) == SHAPE_WAVE:
        k = 2.0 * math.pi * int(p["pert_mode"]) / (g.n[0] * g.h)
        yi = p["R"] * (1.0 - float(p["pert_amp"]) * np.cos(k * (X[0] - 0.5 * g.h)))
        return 0.5 * (1.0 + np.tanh((yi - X[1]) / (2.0 * p["eps"])))
    rel = [X[d] - 0.5 * g.n[d] * g.h for d in range(g.dim)]
    r = np.sqrt(sum(v * v for v in rel))
    R = p["R"]
    m, a = int(p.get("pert_mode", 0)), float(p.get("pert_amp", 0.0))
    if m > 0 and a != 0.0:
        if g.dim == 2:
            theta = np.arctan2(rel[1], rel[0])
            Rt = R * (1.0 + a * np.cos(m * theta))
        else:
            safe = np.where(r > 0.0, r, 1.0)
            ct = np.where(r > 0.0, rel[2] / safe, 1.0)
            Rt = R * (1.0 + a * eval_legendre(m, ct))
    else:
        Rt = R * np.ones_like(r)
    return 0.5 * (1.0 + np.tanh((Rt - r) / (2.0 * p["eps"])))


# ----------------------------------------------------------------------------
# cell-centred operators
# ----------------------------------------------------------------------------
def grad_c(phi, g):
    """Central cell gradient (phi_{i+1} - phi_{i-1}) / (2h) per direction."""
    return [(S(phi, g, d, 1) - S(phi, g, d, -1)) / (2.0 * g.h) for d in range(g.dim)]


def lap(phi, g):
    """Compact Laplacian sum_d (phi_{i+1} - 2 phi_i + phi_{i-1}) / h^2."""
    out = np.zeros_like(phi)
    for d in range(g.dim):
        out = out + (S(phi, g, d, 1) - 2.0 * phi + S(phi, g, d, -1)) / (g.h * g.h)
    return out


def normals(phi, g, delta_n):
    """Cell normal n = grad phi / (|grad phi| + delta_n) (Table 1 caption), central gradient."""
    gr = grad_c(phi, g)
    mag = np.sqrt(sum(v * v for v in gr))
    return [v / (mag + delta_n) for v in gr], mag


def curvature(phi, g, delta_n):
    """kappa = -div(grad phi / |grad phi|) (Eq. curvature), central divergence of cell normals."""
    n, _ = normals(phi, g, delta_n)
    k = np.zeros_like(phi)
    for d in range(g.dim):
        k = k + (S(n[d], g, d, 1) - S(n[d], g, d, -1)) / (2.0 * g.h)
    return -k


def psi(phi):
    """Double-well free energy psi = [phi (1 - phi)]^2 / 2 (Eq. ac_mu)."""
    return 0.5 * (phi * (1.0 - phi)) ** 2


def dpsi(phi):
    """psi' = phi (1 - phi) (1 - 2 phi) (Eq. ac_mu)."""
    return phi * (1.0 - phi) * (1.0 - 2.0 * phi)


def chem_potential(phi, g, sigma, eps):
    """mu = (sigma_hat / eps) psi' - sigma_hat eps lap(phi), sigma_hat = 6 sigma (Eq. ac_mu)."""
    sh = 6.0 * sigma
    return (sh / eps) * dpsi(phi) - sh * eps * lap(phi, g)


# ----------------------------------------------------------------------------
# face helpers: face i - 1/2 along d is stored at index i
# ----------------------------------------------------------------------------
def face_avg(q, g, d):
    """Two-cell average at the d-face: (q_i + q_{i-1}) / 2."""
    return 0.5 * (q + S(q, g, d, -1))


def face_diff(q, g, d):
    """Face difference (q_i - q_{i-1}) / h."""
    return (q - S(q, g, d, -1)) / g.h


def density_cells(phi, p):
    """rho = rho_out + (rho_in - rho_out) clip(phi, 0, 1) (linear mixing, phi = 1 is the drop)."""
    return p["rho_out"] + (p["rho_in"] - p["rho_out"]) * np.clip(phi, 0.0, 1.0)


def viscosity_cells(phi, p):
    """Dynamic viscosity, linear in clip(phi, 0, 1)."""
    return p["mu_out"] + (p["mu_in"] - p["mu_out"]) * np.clip(phi, 0.0, 1.0)


def face_beta(phi, g, p):
    """Face coefficients 1 / rho_f with rho_f the two-cell mean of cell densities."""
    rc = density_cells(phi, p)
    return [1.0 / face_avg(rc, g, d) for d in range(g.dim)]


# ----------------------------------------------------------------------------
# ACDI: the accurate conservative diffuse-interface model (Jain, J. Comput.
# Phys. 469, 2022), the model the 256^2 and 384^3 workloads name; this paper
# does not define it. Same flux form as CDI with the sharpening term evaluated
# through the signed-distance-like variable psi.
# ----------------------------------------------------------------------------
ACDI_EPS0 = 1e-20


def acdi_psi(phi, eps):
    """psi = eps ln((phi + eps0) / (1 - phi + eps0)) of clip(phi, 0, 1), eps0 = 1e-20.

    For the equilibrium profile phi = [1 + tanh(s / (2 eps))] / 2 this is the
    signed distance s (up to eps0); eps0 keeps it finite where phi is 0 or 1
    (|psi| <= 46.1 eps), and the clip keeps the logarithm real (reading).
    """
    p = np.clip(phi, 0.0, 1.0)
    return eps * np.log((p + ACDI_EPS0) / (1.0 - p + ACDI_EPS0))


def acdi_sharpening(psi_f, eps):
    """The ACDI sharpening coefficient (1/4) [1 - tanh^2(psi_f / (2 eps))]: phi (1 - phi)
    of the equilibrium profile at the signed distance psi_f."""
    t = np.tanh(psi_f / (2.0 * eps))
    return 0.25 * (1.0 - t * t)


# ----------------------------------------------------------------------------
# phase-field right-hand side (Eq. 1 with g from Table 1)
# ----------------------------------------------------------------------------
def phase_rhs(phi, u, g, p, gamma):
    """d phi / dt = -div(u phi) + g(phi) for the CDI, SB or ISODI model (Table 1).

    CDI is written in flux form: the d-face flux is
      F = u phi_f - gamma [eps (phi_i - phi_{i-1}) / h - phi_f (1 - phi_f) n_f]
    with phi_f, n_f two-cell averages, and the right-hand side is -sum_d dF/dx_d.
    SB adds gamma [eps lap(phi) - psi'/eps + eps |grad phi| kappa] and ISODI
    gamma [eps lap(phi) - psi'/eps + phi (1 - phi) kappa] to the same
    conservative central advective term.
    ACDI (Jain 2022; not in this paper) has the CDI flux with the sharpening
    term (1/4) [1 - tanh^2(psi_f / (2 eps))] n_f, psi = acdi_psi(phi), psi_f
    the two-cell average and n the cell normals of psi, two-cell averaged.
    """
    eps, dn = p["eps"], p["delta_n"]
    model = p["model"]
    rhs = np.zeros_like(phi)
    if model in (MODEL_CDI, MODEL_ACDI):
        if model == MODEL_ACDI:
            psi = acdi_psi(phi, eps)
            n, _ = normals(psi, g, dn)
        else:
            n, _ = normals(phi, g, dn)
        for d in range(g.dim):
            pf = face_avg(phi, g, d)
            nf = face_avg(n[d], g, d)
            if model == MODEL_ACDI:
                sharp = acdi_sharpening(face_avg(psi, g, d), eps)
            else:
                sharp = pf * (1.0 - pf)
            F = u[d] * pf - gamma * (eps * face_diff(phi, g, d) - sharp * nf)
            rhs = rhs - (S(F, g, d, 1) - F) / g.h
        return rhs
    for d in range(g.dim):
        F = u[d] * face_avg(phi, g, d)
        rhs = rhs - (S(F, g, d, 1) - F) / g.h
    kap = curvature(phi, g, dn)
    if model == MODEL_SB:
        _, mag = normals(phi, g, dn)
        third = eps * mag * kap
    elif model == MODEL_ISODI:
        third = phi * (1.0 - phi) * kap
    else:
        raise ValueError("unknown phase-field model")
    return rhs + gamma * (eps * lap(phi, g) - dpsi(phi) / eps + third)


# ----------------------------------------------------------------------------
# surface tension forces at faces
# ----------------------------------------------------------------------------
def surface_force(phi, g, p):
    """Face force per unit volume for the chosen model.

    EB   (Eq. eb_st):    F = mu_f (phi_i - phi_{i-1}) / h, mu the chemical potential;
    CSF  (Section 2):    F = sigma kappa_f (phi_i - phi_{i-1}) / h;
    LCSF (Eq. equivalence, Section 2.2):
                         F = 6 sigma kappa_f phi_f (1 - phi_f) (phi_i - phi_{i-1}) / h.
    All use the same face gradient as the pressure (balanced force); the force
    enters the momentum right-hand side with a positive sign (Section 2).
    """
    force = p["force"]
    sigma, eps, dn = p["sigma"], p["eps"], p["delta_n"]
    out = []
    if force == FORCE_EB:
        mu = chem_potential(phi, g, sigma, eps)
        for d in range(g.dim):
            out.append(face_avg(mu, g, d) * face_diff(phi, g, d))
        return out
    kap = curvature(phi, g, dn)
    for d in range(g.dim):
        kf = face_avg(kap, g, d)
        if force == FORCE_CSF:
            out.append(sigma * kf * face_diff(phi, g, d))
        elif force == FORCE_LCSF:
            pf = face_avg(phi, g, d)
            out.append(6.0 * sigma * kf * pf * (1.0 - pf) * face_diff(phi, g, d))
        else:
            raise ValueError("unknown force model")
    return out


# ----------------------------------------------------------------------------
# momentum right-hand side (no pressure)
# ----------------------------------------------------------------------------
def transverse_velocity(u, g, d, e):
    """Component e interpolated to the d-faces: mean of the four e-faces around it."""
    ue = u[e]
    return 0.25 * (ue + S(ue, g, e, 1) + S(ue, g, d, -1) + S(S(ue, g, d, -1), g, e, 1))


def momentum_rhs(phi, u, g, p):
    """du_d/dt without pressure on the d-faces:
       -(u . grad) u_d + (1/rho_f) div(eta (grad u + grad u^T))_d + F_d / rho_f.

    Advection: central differences of u_d with the transverse components
    averaged from four faces. Viscous stress: tau_dd = 2 eta (u_d(i+1) - u_d(i))/h
    at cell centres, tau_de = eta_edge (du_d/dx_e + du_e/dx_d) at the edge
    (i - e_d/2 - e_e/2), eta_edge the mean of the four cells around the edge.
    The paper gives only the force; this form is a reading (Section 3 defers it).
    """
    h = g.h
    eta = viscosity_cells(phi, p)
    beta = face_beta(phi, g, p)
    F = surface_force(phi, g, p)
    out = []
    for d in range(g.dim):
        ud = u[d]
        adv = np.zeros_like(ud)
        for e in range(g.dim):
            vel = ud if e == d else transverse_velocity(u, g, d, e)
            adv = adv + vel * (S(ud, g, e, 1) - S(ud, g, e, -1)) / (2.0 * h)
        visc = np.zeros_like(ud)
        for e in range(g.dim):
            if e == d:
                tau = 2.0 * eta * (S(ud, g, d, 1) - ud) / h
                visc = visc + (tau - S(tau, g, d, -1)) / h
            else:
                eta_e = 0.25 * (eta + S(eta, g, d, -1) + S(eta, g, e, -1)
                                + S(S(eta, g, d, -1), g, e, -1))
                tau = eta_e * ((ud - S(ud, g, e, -1)) / h + (u[e] - S(u[e], g, d, -1)) / h)
                visc = visc + (S(tau, g, e, 1) - tau) / h
        out.append(-adv + beta[d] * visc + beta[d] * F[d])
    return out


# ----------------------------------------------------------------------------
# consistent (conservative) momentum transport
# ----------------------------------------------------------------------------
def cdi_face_flux(phi, u, g, p, gamma, d):
    """CDI flux through the d-faces, u phi_f - gamma [eps dphi - phi_f (1 - phi_f) n_f]
    (the flux whose divergence is the CDI phase-field right-hand side, Table 1)."""
    n, _ = normals(phi, g, p["delta_n"])
    pf = face_avg(phi, g, d)
    nf = face_avg(n[d], g, d)
    return u[d] * pf - gamma * (p["eps"] * face_diff(phi, g, d) - pf * (1.0 - pf) * nf)


def mass_flux(phi, u, g, p, gamma):
    """Mass flux through the d-faces consistent with the CDI phase field.

    With rho = rho_out + (rho_in - rho_out) phi and d phi/dt = -sum_d dF_d/dx_d,
    the density obeys d rho/dt = -sum_d dm_d/dx_d with
    m_d = rho_out u_d + (rho_in - rho_out) F_d (exactly, where 0 <= phi <= 1).
    """
    drho = p["rho_in"] - p["rho_out"]
    return [p["rho_out"] * u[d] + drho * cdi_face_flux(phi, u, g, p, gamma, d)
            for d in range(g.dim)]


def momentum_rhs_consistent(phi, u, g, p, gamma):
    """d(rho_f u_d)/dt without pressure on the d-faces, conservative form:
       -div(m u_d) + div(eta (grad u + grad u^T))_d + F_d,
    m the mass flux consistent with the phase field (mass_flux).

    The momentum flux of u_d along d lives at cell centres: mean of m_d over the
    cell's two d-faces times the mean of u_d over them. Along e != d it lives at
    the edge between cells i, i-d, i-e, i-d-e: mean of m_e over the e-faces of
    cells i and i-d times the mean of u_d over the d-faces of cells i and i-e.
    The viscous stress and the surface force are those of momentum_rhs, not
    divided by rho_f. The paper defers this transport to its reference
    [Mirjalili 2021]; this discrete form is a reading.
    """
    if p["model"] != MODEL_CDI:
        raise ValueError("consistent momentum transport needs the CDI model")
    h = g.h
    m = mass_flux(phi, u, g, p, gamma)
    eta = viscosity_cells(phi, p)
    F = surface_force(phi, g, p)
    out = []
    for d in range(g.dim):
        ud = u[d]
        adv = np.zeros_like(ud)
        for e in range(g.dim):
            if e == d:
                flux = 0.5 * (m[d] + S(m[d], g, d, 1)) * 0.5 * (ud + S(ud, g, d, 1))
                adv = adv + (flux - S(flux, g, d, -1)) / h
            else:
                flux = 0.5 * (m[e] + S(m[e], g, d, -1)) * 0.5 * (ud + S(ud, g, e, -1))
                adv = adv + (S(flux, g, e, 1) - flux) / h
        visc = np.zeros_like(ud)
        for e in range(g.dim):
            if e == d:
                tau = 2.0 * eta * (S(ud, g, d, 1) - ud) / h
                visc = visc + (tau - S(tau, g, d, -1)) / h
            else:
                eta_e = 0.25 * (eta + S(eta, g, d, -1) + S(eta, g, e, -1)
                                + S(S(eta, g, d, -1), g, e, -1))
                tau = eta_e * ((ud - S(ud, g, e, -1)) / h + (u[e] - S(u[e], g, d, -1)) / h)
                visc = visc + (S(tau, g, e, 1) - tau) / h
        out.append(-adv + visc + F[d])
    return out


def face_density(phi, g, p):
    """rho_f on the d-faces: the two-cell mean of the cell densities."""
    rc = density_cells(phi, p)
    return [face_avg(rc, g, d) for d in range(g.dim)]


# ----------------------------------------------------------------------------
# projection
# ----------------------------------------------------------------------------
def divergence(u, g):
    """(D u)_i = sum_d (u_d(i+1) - u_d(i)) / h at cell centres."""
    out = np.zeros(g.shape)
    for d in range(g.dim):
        out = out + (S(u[d], g, d, 1) - u[d]) / g.h
    return out


def gradient_faces(q, g):
    """(G q)_d = (q_i - q_{i-1}) / h on the d-faces; G = -D^T."""
    return [face_diff(q, g, d) for d in range(g.dim)]


def poisson_matrix(beta, g):
    """Sparse A = -D diag(beta) G, symmetric positive semidefinite, A 1 = 0."""
    N = int(np.prod(g.shape))
    idx = np.arange(N).reshape(g.shape)
    rows, cols, vals = [], [], []
    for d in range(g.dim):
        w = (beta[d] / (g.h * g.h)).ravel()
        a = idx.ravel()
        b = S(idx, g, d, -1).ravel()
        rows += [a, b, a, b]
        cols += [a, b, b, a]
        vals += [w, w, -w, -w]
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A


def apply_poisson(beta, q, g):
    """A q = -D(beta G q) evaluated with stencils (same operator as poisson_matrix)."""
    G = gradient_faces(q, g)
    return -divergence([beta[d] * G[d] for d in range(g.dim)], g)


def solve_poisson(beta, rhs, g):
    """Exact solution of A x = rhs with mean(x) = 0 (rhs projected to zero mean).

    The singular periodic system is made regular by pinning cell 0 and then
    removing the mean; SuperLU factorizes the reduced matrix (minimum-degree
    ordering of A^T + A, which suits this symmetric stencil matrix: the fill,
    and so the time, of a 3D factorization is a third of the column ordering's).
    """
    A = poisson_matrix(beta, g)
    b = (rhs - rhs.mean()).ravel()
    Ar = A[1:, 1:].tocsc()
    x = np.zeros_like(b)
    x[1:] = spla.spsolve(Ar, b[1:], permc_spec="MMD_AT_PLUS_A")
    x = x - x.mean()
    return x.reshape(g.shape)


def pressure_beta(phi, g, p):
    """Face coefficients of the projection: 1 / rho_f, and 0 on the wall faces
    when walls bound the box in y (no flux through a wall: the homogeneous
    Neumann condition of the pressure there)."""
    beta = face_beta(phi, g, p)
    if p.get("wall_y", 0):
        beta[1] = beta[1].copy()
        _wall_rows(beta[1], g)[...] = 0.0
    return beta


def project(ustar, phi, g, p, tau):
    """u = u* - tau beta G p with D(beta G p) = D u* / tau, mean(p) = 0.

    The pressure solves A p = -b, A = -D beta G, b = D u* / tau projected to
    zero mean; p is the physical pressure of the stage. Between walls in y the
    wall faces carry beta = 0, so p obeys dp/dn = 0 there and the wall's
    normal velocity (zero in u*) is not corrected.
    """
    beta = pressure_beta(phi, g, p)
    b = divergence(ustar, g) / tau
    b = b - b.mean()
    pr = solve_poisson(beta, -b, g)
    Gp = gradient_faces(pr, g)
    u = [ustar[d] - tau * beta[d] * Gp[d] for d in range(g.dim)]
    return u, pr


# ----------------------------------------------------------------------------
# free-slip walls in y (Section 3.2 standing wave: periodic in x, free slip on
# the top and bottom walls)
# ----------------------------------------------------------------------------
# The walls lie at y = 0 and y = ny h, on the y-face of index 0 (face ny wraps
# to it). Free slip: zero normal velocity and zero tangential stress; with no
# flux of phi through a wall and phi of zero normal gradient there. The
# right-hand sides are evaluated on the box extended by WALL_GHOST image rows
# beyond each wall: cell-centred quantities (phi, the x-velocity) mirror
# (cell -1-j is cell j), the y-velocity is odd about the wall faces
# (v(-j) = -v(j), v(ny) = 0). Every stencil then sees a zero normal gradient
# of phi, a zero normal velocity and a zero shear du/dy at the walls; normals,
# chemical potential and curvature computed from the images carry the right
# parity by construction. Stencils reach at most three cells.
WALL_GHOST = 3


def _wall_rows(a, g):
    """View of the y-face row 0 (the wall faces) of a face array."""
    return np.moveaxis(a, g.axis(1), 0)[0]


def _pad_y(a, g, odd_face):
    """a extended by WALL_GHOST image rows below y = 0 and above y = ny h."""
    G = WALL_GHOST
    b = np.moveaxis(a, g.axis(1), 0)
    ny = b.shape[0]
    if odd_face:
        lo = -b[G:0:-1]                                                   # faces -G .. -1
        hi = np.concatenate([np.zeros_like(b[:1]), -b[ny - 1:ny - G:-1]])  # faces ny .. ny+G-1
    else:
        lo = b[G - 1::-1]                                                 # cells -G .. -1
        hi = b[ny - 1:ny - 1 - G:-1]                                      # cells ny .. ny+G-1
    return np.moveaxis(np.concatenate([lo, b, hi]), 0, g.axis(1))


def _crop_y(a, g):
    """The rows of the box proper from an array on the extended box."""
    b = np.moveaxis(a, g.axis(1), 0)
    return np.moveaxis(b[WALL_GHOST:b.shape[0] - WALL_GHOST], 0, g.axis(1))


def _extended(phi, u, g):
    n = list(g.n)
    n[1] += 2 * WALL_GHOST
    ge = Grid(g.dim, n, g.L)
    ue = [_pad_y(u[d], g, odd_face=(d == 1)) for d in range(g.dim)]
    return ge, _pad_y(phi, g, False), ue


def phase_rhs_walls(phi, u, g, p, gamma):
    """phase_rhs between free-slip walls in y (image rows beyond the walls)."""
    ge, phie, ue = _extended(phi, u, g)
    return _crop_y(phase_rhs(phie, ue, ge, p, gamma), g)


def momentum_rhs_walls(phi, u, g, p):
    """momentum_rhs between free-slip walls in y; the wall's normal velocity
    has no right-hand side (it stays zero)."""
    ge, phie, ue = _extended(phi, u, g)
    k = [_crop_y(c, g) for c in momentum_rhs(phie, ue, ge, p)]
    k[1] = k[1].copy()
    _wall_rows(k[1], g)[...] = 0.0
    return k


# ----------------------------------------------------------------------------
# time step
# ----------------------------------------------------------------------------
def gamma_of(u, p):
    """Gamma = gamma_fixed if set, else max(gamma_min, max |u| over all faces)."""
    if p.get("gamma_fixed", 0.0) > 0.0:
        return float(p["gamma_fixed"])
    um = max(float(np.max(np.abs(c))) for c in u) if u else 0.0
    return max(float(p.get("gamma_min", 0.0)), um)


class State:
    def __init__(self, phi, u, pr, step=0, t=0.0):
        self.phi, self.u, self.p, self.step, self.t = phi, u, pr, step, t

    def copy(self):
        return State(self.phi.copy(), [c.copy() for c in self.u], self.p.copy(), self.step, self.t)


def initial_state(p, phi0=None):
    g = Grid(p["dim"], p["n"], p["L"])
    phi = initial_phi(p) if phi0 is None else np.array(phi0, dtype=np.float64).reshape(g.shape)
    u = [np.zeros(g.shape) for _ in range(g.dim)]
    return State(phi, u, np.zeros(g.shape))


def step(st, p):
    """One time step: projected RK4 (Section 3: RK4 in time) or forward Euler.

    RK4: stage s evaluates k_s = (rhs_phi, rhs_u) at (phi_s, u_s); the next
    stage is phi_{s+1} = phi^n + c_{s+1} dt k_s, u_{s+1} = P(u^n + c_{s+1} dt k_s)
    projected with rho(phi_{s+1}); the step ends with
    phi^{n+1} = phi^n + dt sum_s w_s k_s and u^{n+1} = P(u^n + dt sum_s w_s k_s).
    Gamma is frozen over the step at its value from u^n. With consistent
    momentum transport (momentum = 1) the stages advance rho_f u instead:
    u_{s+1} = P((rho_f^n u^n + c_{s+1} dt k_s) / rho_f(phi_{s+1})), likewise at the end.
    """
    p = params_from(p)
    g = Grid(p["dim"], p["n"], p["L"])
    dt = p["dt"]
    gam = gamma_of(st.u, p)
    phin, un = st.phi, st.u
    cons = p.get("momentum", MOMENTUM_ADVECTIVE) == MOMENTUM_CONSISTENT
    walls = bool(p.get("wall_y", 0))
    if walls and (cons or g.dim != 2):
        raise ValueError("walls in y: 2D with advective momentum transport")

    def prhs(ph, uu):
        return phase_rhs_walls(ph, uu, g, p, gam) if walls else phase_rhs(ph, uu, g, p, gam)

    if cons:
        # consistent transport advances rho_f u: the stage velocity is the new
        # momentum divided by the face density of the new phase field
        rn = face_density(phin, g, p)
        vn = [rn[d] * un[d] for d in range(g.dim)]

        def krhs(ph, uu):
            return momentum_rhs_consistent(ph, uu, g, p, gam)

        def vel(v, ph):
            r = face_density(ph, g, p)
            return [v[d] / r[d] for d in range(g.dim)]
    else:
        vn = un

        def krhs(ph, uu):
            return momentum_rhs_walls(ph, uu, g, p) if walls else momentum_rhs(ph, uu, g, p)

        def vel(v, ph):
            return v
    if p["scheme"] == SCHEME_FE:
        kphi = prhs(phin, un)
        ku = krhs(phin, un)
        phi1 = phin + dt * kphi
        ustar = vel([vn[d] + dt * ku[d] for d in range(g.dim)], phi1)
        u1, pr = project(ustar, phi1, g, p, dt)
        return State(phi1, u1, pr, st.step + 1, st.t + dt)
    phis, us = phin, un
    acc_phi = None
    acc_u = None
    pr = st.p
    for s in range(4):
        kphi = prhs(phis, us)
        ku = krhs(phis, us)
        wdt = RK4_W[s] * dt
        if s < 3:
            acc_phi = wdt * kphi if s == 0 else acc_phi + wdt * kphi
            acc_u = [wdt * ku[d] if s == 0 else acc_u[d] + wdt * ku[d] for d in range(g.dim)]
            cdt = RK4_C[s + 1] * dt
            phis = phin + cdt * kphi
            ustar = vel([vn[d] + cdt * ku[d] for d in range(g.dim)], phis)
            us, pr = project(ustar, phis, g, p, cdt)
        else:
            phi_new = phin + (acc_phi + wdt * kphi)
            ustar = vel([vn[d] + (acc_u[d] + wdt * ku[d]) for d in range(g.dim)], phi_new)
            u_new, pr = project(ustar, phi_new, g, p, dt)
            return State(phi_new, u_new, pr, st.step + 1, st.t + dt)


def timed_run(job):
    """(params, steps) -> (cells x steps, seconds): steps of the oracle from the
    initial state, timed (a task of the host baseline's process pool; params
    None is a no-op that warms a worker)."""
    import time

    p, steps = job
    if p is None:
        return 0, 0.0
    p = params_from(dict(p, precision="fp64"))
    st = initial_state(p)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = step(st, p)
    return int(np.prod(Grid(p["dim"], p["n"], p["L"]).shape)) * steps, time.perf_counter() - t0


def run(p, steps=None, phi0=None, record=False):
    p = params_from(p)
    st = initial_state(p, phi0)
    hist = []
    nsteps = p["steps"] if steps is None else steps
    for _ in range(nsteps):
        st = step(st, p)
        if record:
            hist.append(diagnostics(st, p))
    return (st, hist) if record else st


# ----------------------------------------------------------------------------
# diagnostics (Section 3.1 Ca_inf, Section 3.2 energies)
# ----------------------------------------------------------------------------
def surface_energy(phi, g, sigma, eps, wall_y=0):
    """SE = sum [ (sigma_hat/eps) psi + (sigma_hat eps / 2) |grad phi|^2 ] dV.

    |grad phi|^2 is the sum of squared face differences, so d SE / d phi_i / dV
    equals the discrete chemical potential. The 1/2 on the gradient term makes
    mu the variational derivative of SE (Eq. ac_mu); the energy formula printed
    in Section 3.2 omits it (reading: a misprint).
    """
    sh = 6.0 * sigma
    terms = [face_diff(phi, g, d) ** 2 for d in range(g.dim)]
    if wall_y:
        _wall_rows(terms[1], g)[...] = 0.0    # phi mirrors across a wall: no jump there
    grad2 = sum(terms)
    return float(np.sum((sh / eps) * psi(phi) + 0.5 * sh * eps * grad2) * g.dV)


def diagnostics(st, p):
    p = params_from(p)
    g = Grid(p["dim"], p["n"], p["L"])
    phi, u, pr = st.phi, st.u, st.p
    rho = density_cells(phi, p)
    ke = 0.0
    for d in range(g.dim):
        ke += 0.5 * float(np.sum(face_avg(rho, g, d) * u[d] ** 2)) * g.dV
    umax = max(float(np.max(np.abs(c))) for c in u)
    inside, outside = phi >= 0.999, phi <= 0.001
    dp = float(pr[inside].mean() - pr[outside].mean()) if inside.any() and outside.any() else 0.0
    return dict(mass=float(np.sum(phi)) * g.dV, ke=ke,
                se=surface_energy(phi, g, p["sigma"], p["eps"], p.get("wall_y", 0)),
                umax=umax, ca_inf=umax * p["mu_in"] / p["sigma"], dp_laplace=dp,
                phi_min=float(phi.min()), phi_max=float(phi.max()), step=st.step, t=st.t)


def laplace_jump_pde(dim, sigma, R, eps, nquad=200001):
    """Pressure jump of the continuum static drop with the EB force.

    Integrating dp/dr = mu dphi/dr across the radial tanh profile, where the
    chemical potential reduces to 6 sigma phi (1 - phi) (d - 1) / r, gives
    dp = int 6 sigma (d - 1) phi^2 (1 - phi)^2 / (eps r) dr (trapezoid rule).
    The tanh profile in R - r has a cusp at r = 0 where the integrand behaves
    like exp(-2R/eps)/r; the integral starts at r = R/1000, which drops a
    contribution of order exp(-2R/eps) (6 (d-1)/eps) log(1000).
    """
    r = np.linspace(1e-3 * R, R + 40.0 * eps, nquad)
    phi = 0.5 * (1.0 + np.tanh((R - r) / (2.0 * eps)))
    f = 6.0 * sigma * (dim - 1) * phi ** 2 * (1.0 - phi) ** 2 / (eps * r)
    return float(np.trapezoid(f, r))


def lamb_frequency(dim, mode, sigma, R, rho_in, rho_out):
    """Linear-theory angular frequency of a mode-n drop oscillation (inviscid)."""
    n = mode
    if dim == 2:
        return math.sqrt(n * (n * n - 1) * sigma / ((rho_in + rho_out) * R ** 3))
    return math.sqrt((n - 1) * n * (n + 1) * (n + 2) * sigma
                     / (R ** 3 * ((n + 1) * rho_in + n * rho_out)))
