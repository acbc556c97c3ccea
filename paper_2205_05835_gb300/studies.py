"""Spurious-current convergence studies of Section 3.1 on the batched executor.

The static-drop benchmark of Section 3.1 (drop of diameter D = 0.4 centred in
the unit box, equal densities rho = 300 and viscosities mu = 0.1, sigma = 1,
Laplace number La = sigma rho D / mu^2 = 12000) is run for every phase-field
model (CDI, SB, ISODI) and surface tension force (EB, CSF, LCSF) on a sequence
of meshes, all instances concurrently in one pf_batch, to the dimensionless
time t* = sigma t / (mu D) = 250; the capillary number of the spurious
currents Ca_inf = max|u| mu / sigma is reported per model, force and mesh
with the observed convergence order between successive meshes.

Two panels (Fig. 2):
  "h"   -- fixed interface thickness eps = 1/32, mesh refined N = 32 ... 256;
  "eps" -- sharp-interface limit: the mesh is doubled and eps is tied to it by
           dx = 32^(1/2) eps^(3/2), i.e. eps = (dx / sqrt 32)^(2/3).

The box is periodic here (the paper's walls are free-slip; the drop is far
from them). The paper's Fig. 2 data are not available, so the output is a
table to compare with the figure's trends (EB second order), not a parity
check.

    python -m paper_2205_05835_gb300.studies --panel h --tstar 250

A second driver compares the forces and the precisions on the density-ratio-
1000 static drop (256^2, rho 240 / 0.24, mu 0.1 / 0.001, CDI, eps = dx):
EB, CSF and LCSF each in float64 and in mixed precision, run concurrently,
reporting the spurious currents, the Laplace pressure jump against sigma / R
and the mixed path's per-field distance from the float64 run of the same force:

    python -m paper_2205_05835_gb300.studies --compare --steps 2000

A third driver runs the standing wave of Section 3.2 (2 pi x 2 pi box,
periodic in x, free-slip walls in y, sigma = 2, rho = 1, nu = 0.064720863,
initial amplitude A0 = 2 pi / 100, one wavelength) for every force on a mesh
sequence at fixed eps = (2 pi) / 32 ("h", Figs. 6 and 7 a-c) or on the
sharp-interface sequence dx = 32^(1/2) eps^(3/2) ("eps", Figs. 6 and 7 d),
and reports the amplitude A(t) / lambda at x = dx/2, its l2 distance from the
viscous initial-value solution of Prosperetti (1981) and the kinetic,
surface and total energy histories (Fig. 8):

    python -m paper_2205_05835_gb300.studies --wave h --ns 16,32,64,128
"""
from __future__ import annotations

import argparse
import json
import math
import time

SIGMA, MU, D, LA = 1.0, 0.1, 0.4, 12000.0


def eps_of(panel, n):
    if panel == "h":
        return 1.0 / 32
    return (1.0 / (n * math.sqrt(32.0))) ** (2.0 / 3.0)


def drop_params(n, model, force, eps, precision="mixed", cfl=0.5):
    """Static-drop instance on an n x n periodic grid; dt is cfl times the
    smallest of the capillary and viscous limits."""
    rho = LA * MU * MU / (SIGMA * D)
    h = 1.0 / n
    dt = cfl * min(math.sqrt(2 * rho * h ** 3 / (4 * math.pi * SIGMA)), h * h * rho / (4 * MU))
    return dict(dim=2, n=(n, n, 1), L=1.0, model=model, force=force, precision=precision,
                scheme="rk4", sigma=SIGMA, eps=eps, rho_in=rho, rho_out=rho, mu_in=MU, mu_out=MU,
                gamma_fixed=0.0, gamma_min=0.0, dt=dt, delta_n=1e-12, poisson_rtol=1e-10,
                poisson_maxit=200, R=D / 2, pert_mode=0, pert_amp=0.0)


def study_instances(panel, ns, models, forces, precision="mixed"):
    plist, keys = [], []
    for m in models:
        for f in forces:
            for n in ns:
                plist.append(drop_params(n, m, f, eps_of(panel, n), precision=precision))
                keys.append((m, f, n))
    return plist, keys


def convergence_study(panel="h", ns=(32, 64, 128, 256), models=("cdi", "sb", "isodi"),
                      forces=("eb", "csf", "lcsf"), tstar=250.0, nthreads=16,
                      precision="mixed"):
    """Ca_inf at t* for every (model, force, mesh); returns the table and the
    observed orders log(Ca(N) / Ca(2N)) / log 2."""
    import paper_2205_05835_gb300 as pf

    plist, keys = study_instances(panel, ns, models, forces, precision)
    bat = pf.Batch(plist, nthreads=nthreads)
    t_end = tstar * MU * D / SIGMA
    steps = [int(math.ceil(t_end / p["dt"])) for p in plist]
    t0 = time.perf_counter()
    bat.step_each(steps)
    wall = time.perf_counter() - t0
    table = {}
    for i, (m, f, n) in enumerate(keys):
        d = bat.diagnostics(i)
        table.setdefault(m, {}).setdefault(f, {})[n] = {"ca_inf": d["ca_inf"], "t": d["t"]}
    bat.close()
    orders = {}
    for m in models:
        for f in forces:
            row = table[m][f]
            o = []
            for a, b in zip(ns[:-1], ns[1:]):
                ca, cb = row[a]["ca_inf"], row[b]["ca_inf"]
                o.append(math.log(ca / cb) / math.log(b / a) if ca > 0 and cb > 0
                         else float("nan"))
            orders[f"{m}-{f}"] = o
    cells_steps = sum(p["n"][0] * p["n"][1] * s for p, s in zip(plist, steps))
    return {"panel": panel, "tstar": tstar, "ns": list(ns),
            "eps": {n: eps_of(panel, n) for n in ns}, "ca_inf": table, "orders": orders,
            "wall_s": wall, "mcell_steps_per_s": cells_steps / wall / 1e6,
            "steps": {f"{m}-{f}-{n}": s for (m, f, n), s in zip(keys, steps)}}


def force_precision_comparison(n=256, steps=2000, forces=("eb", "csf", "lcsf"),
                               use_graph=1):
    """The static drop at density ratio 1000 for every force in float64 and
    mixed precision (one batch); per force: Ca_inf, Laplace jump dp and its
    relative deviation from sigma / R in both precisions (after the first step,
    the pressure balancing the initial equilibrium profile, and at the end),
    and the max-norm relative distance of the mixed fields from the float64
    fields."""
    import numpy as np

    import paper_2205_05835_gb300 as pf
    import pf_inputs as I

    plist, keys = [], []
    for f in forces:
        for prec in ("fp64", "mixed"):
            p = I.static_drop_256_r1000(force=f, precision=prec)
            p["n"] = (n, n, 1)
            p["eps"] = None
            p["dt"] = None
            p = I.finalize(p)
            p["use_graph"] = use_graph
            plist.append(p)
            keys.append((f, prec))
    bat = pf.Batch(plist)
    t0 = time.perf_counter()
    bat.step(1)
    dp1 = [bat.diagnostics(i)["dp_laplace"] for i in range(len(plist))]
    bat.step(steps - 1)
    wall = time.perf_counter() - t0
    out = {"n": n, "steps": steps, "wall_s": wall, "forces": {}}
    for f in forces:
        i64, i32 = keys.index((f, "fp64")), keys.index((f, "mixed"))
        row = {}
        for prec, i in (("fp64", i64), ("mixed", i32)):
            d = bat.diagnostics(i)
            ref = plist[i]["sigma"] / plist[i]["R"]
            row[prec] = {"ca_inf": d["ca_inf"], "dp": d["dp_laplace"],
                         "dp_rel_to_sigma_over_R": d["dp_laplace"] / ref - 1.0,
                         "dp_first_step_rel": dp1[i] / ref - 1.0,
                         "mass": d["mass"], "phi_min": d["phi_min"], "phi_max": d["phi_max"],
                         "t": d["t"]}
        errs = {}
        for name in ("phi", "u", "v", "p"):
            a, b = bat.field(i64, name), bat.field(i32, name)
            errs[name] = float(np.max(np.abs(b - a)) / max(float(np.max(np.abs(a))), 1e-300))
        row["mixed_vs_fp64"] = errs
        out["forces"][f] = row
    bat.close()
    return out


def prosperetti_amplitude(t, k, nu, sigma, rho1, rho2):
    """Amplitude a(t) / a(0) of a small capillary wave of wavenumber k between
    two unbounded fluids of equal kinematic viscosity nu, released from rest
    (Prosperetti 1981, the exact solution the paper's Section 3.2 compares
    with):

      a / a0 = 4 (1 - 4 b) nu^2 k^4 / (8 (1 - 4 b) nu^2 k^4 + w0^2) erfc(sqrt(nu k^2 t))
               + sum_i z_i w0^2 / (Z_i (z_i^2 - nu k^2)) exp((z_i^2 - nu k^2) t) erfc(z_i sqrt t)

    with b = rho1 rho2 / (rho1 + rho2)^2, w0^2 = sigma k^3 / (rho1 + rho2),
    z_i the four roots of
      z^4 - 4 b (k^2 nu)^(1/2) z^3 + 2 (1 - 6 b) k^2 nu z^2
          + 4 (1 - 3 b) (k^2 nu)^(3/2) z + (1 - 4 b) nu^2 k^4 + w0^2 = 0
    and Z_i = prod_{j != i} (z_j - z_i). exp(z^2 t) erfc(z sqrt t) is
    evaluated as the scaled complementary error function w(i z sqrt t)
    (Faddeeva), which stays finite where the two factors would not.
    """
    import numpy as np
    from scipy.special import erfc, wofz

    b = rho1 * rho2 / (rho1 + rho2) ** 2
    w02 = sigma * k ** 3 / (rho1 + rho2)
    nk = k * k * nu
    z = np.roots([1.0, -4.0 * b * math.sqrt(nk), 2.0 * (1.0 - 6.0 * b) * nk,
                  4.0 * (1.0 - 3.0 * b) * nk ** 1.5, (1.0 - 4.0 * b) * nk * nk + w02])
    t = np.asarray(t, dtype=np.float64)
    a = (4.0 * (1.0 - 4.0 * b) * nk * nk / (8.0 * (1.0 - 4.0 * b) * nk * nk + w02)
         * erfc(np.sqrt(nk * t))).astype(np.complex128)
    for i in range(4):
        Zi = np.prod([z[j] - z[i] for j in range(4) if j != i])
        a = a + z[i] * w02 / (Zi * (z[i] ** 2 - nk)) * np.exp(-nk * t) * wofz(1j * z[i] * np.sqrt(t))
    return a.real


def wave_eps(panel, n):
    """Interface thickness of the standing-wave study on an n x n mesh of the
    2 pi box: eps = 2 pi / 32 ("h"), or dx = 32^(1/2) eps^(3/2) in units of the
    box edge ("eps")."""
    L = 2.0 * math.pi
    if panel == "h":
        return L / 32.0
    return L * (1.0 / (n * math.sqrt(32.0))) ** (2.0 / 3.0)


def standing_wave_study(panel="h", ns=(16, 32, 64, 128), forces=("eb", "csf", "lcsf"),
                        model="cdi", t_end=10.0, sample_dt=0.03, precision="fp64",
                        use_graph=1):
    """Every force on every mesh as one batch; per instance the amplitude
    history A(t) / lambda at x = dx/2 (A = y0 minus the column integral of phi),
    its l2 distance from prosperetti_amplitude over the samples, and the
    KE / SE / TE histories."""
    import numpy as np

    import paper_2205_05835_gb300 as pf
    import pf_inputs as I

    plist, keys = [], []
    for f in forces:
        for n in ns:
            p = I.standing_wave(n=n, force=f, model=model, precision=precision,
                                eps_frac=wave_eps(panel, n) / (2.0 * math.pi))
            p["use_graph"] = use_graph
            plist.append(p)
            keys.append((f, n))
    bat = pf.Batch(plist)
    lam = 2.0 * math.pi
    every = [max(1, int(round(sample_dt / p["dt"]))) for p in plist]
    nsamp = int(math.ceil(t_end / sample_dt))
    hist = [{"t": [], "A": [], "ke": [], "se": []} for _ in plist]

    def sample():
        for i, p in enumerate(plist):
            h = p["L"] / p["n"][0]
            col = float(np.sum(bat.field(i, "phi")[:, 0])) * h
            d = bat.diagnostics(i)
            hist[i]["t"].append(d["t"])
            hist[i]["A"].append((p["R"] - col) / lam)
            hist[i]["ke"].append(d["ke"])
            hist[i]["se"].append(d["se"])

    t0 = time.perf_counter()
    sample()
    for _ in range(nsamp):
        bat.step_each(every)
        sample()
    wall = time.perf_counter() - t0
    bat.close()
    out = {"panel": panel, "model": model, "precision": precision, "t_end": t_end,
           "wall_s": wall, "ns": list(ns), "eps": {n: wave_eps(panel, n) for n in ns},
           "l2": {}, "first_zero": {}, "runs": {}}
    A0 = 2.0 * math.pi / 100.0
    for i, (f, n) in enumerate(keys):
        t = np.array(hist[i]["t"])
        A = np.array(hist[i]["A"])
        ex = A0 / lam * prosperetti_amplitude(t, 1.0, plist[i]["mu_in"], plist[i]["sigma"],
                                              1.0, 1.0)
        l2 = float(np.sqrt(np.mean((A[1:] - ex[1:]) ** 2)))
        zc = np.where((A[:-1] >= 0) & (A[1:] < 0))[0]
        tz = float(t[zc[0]] - A[zc[0]] * (t[zc[0] + 1] - t[zc[0]]) / (A[zc[0] + 1] - A[zc[0]])) \
            if len(zc) else float("nan")
        out["l2"].setdefault(f, {})[n] = l2
        out["first_zero"].setdefault(f, {})[n] = tz
        ke, se = np.array(hist[i]["ke"]), np.array(hist[i]["se"])
        out["runs"][f"{f}-{n}"] = {"dt": plist[i]["dt"], "t": t.tolist(), "A_over_lambda": A.tolist(),
                                    "exact": ex.tolist(), "ke": ke.tolist(), "se": se.tolist(),
                                    "te": (ke + se).tolist()}
    t_ex = np.linspace(0.0, t_end, 200001)
    a_ex = prosperetti_amplitude(t_ex, 1.0, 0.064720863, 2.0, 1.0, 1.0)
    z = np.where((a_ex[:-1] >= 0) & (a_ex[1:] < 0))[0]
    out["first_zero_exact"] = float(t_ex[z[0]]) if len(z) else float("nan")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--panel", choices=("h", "eps"), default="h")
    ap.add_argument("--tstar", type=float, default=250.0)
    ap.add_argument("--ns", type=str, default="32,64,128,256")
    ap.add_argument("--models", type=str, default="cdi,sb,isodi")
    ap.add_argument("--forces", type=str, default="eb,csf,lcsf")
    ap.add_argument("--precision", type=str, default="mixed")
    ap.add_argument("--threads", type=int, default=16)
    ap.add_argument("--compare", action="store_true",
                    help="forces x precisions on the density-ratio-1000 drop")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--wave", choices=("h", "eps"), default=None,
                    help="standing wave (Section 3.2) on the given mesh sequence")
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--wave-precision", default="fp64")
    ap.add_argument("--full", action="store_true", help="include the histories in the output")
    args = ap.parse_args()
    if args.wave:
        res = standing_wave_study(panel=args.wave, ns=tuple(int(v) for v in args.ns.split(",")),
                                  forces=tuple(args.forces.split(",")),
                                  model=args.models.split(",")[0], t_end=args.t_end,
                                  precision=args.wave_precision)
        if not args.full:
            res.pop("runs")
        print(json.dumps(res))
        return
    if args.compare:
        print(json.dumps(force_precision_comparison(n=args.n, steps=args.steps)))
        return
    res = convergence_study(panel=args.panel, ns=tuple(int(v) for v in args.ns.split(",")),
                            models=tuple(args.models.split(",")),
                            forces=tuple(args.forces.split(",")), tstar=args.tstar,
                            nthreads=args.threads, precision=args.precision)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
