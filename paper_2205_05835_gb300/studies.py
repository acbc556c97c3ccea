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
    args = ap.parse_args()
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
