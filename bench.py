"""Throughput of the fractional step (pf_step) on one GB300, in Mcell-steps/s.

Default workload: the 384^3 mode-2 oscillating drop (density and viscosity
ratio 10, ACDI phase field + energy-based force, mixed precision: float32 stencils and
V-cycles inside a refinement to float64 accuracy). One timed step is one
pf_step: four RK stages, each with its phase-field/momentum stage kernels and
one variable-coefficient Poisson solve; by default (--graph 1) each step is
one replayed CUDA graph whose solver loops are device-driven. The state
(~1.4 GB) is far larger than L2, so no flush is needed between steps.

The JSON line also carries: the roofline of the dominant kernel class (timed
with CUDA events inside the library's tracing hooks, in a host-driven pass of
the same steps when the headline runs as graph replays), a whole-step figure
(compulsory bytes of every finest-grid kernel class over the headline time,
a lower bound that leaves out the coarse multigrid levels), an end-to-end
number through the C ABI with the state copied from and to pinned host memory
every step, the FP64 oracle timed on the host cores on a bounded sample, the
SM clocks sampled during the timed region and the number of kernel launches.
Before the timed region the multigrid launch shape (coarse-solve threshold,
smoothing sweeps) is autotuned on the workload's grid, per grid size for the
batch (`--autotune 0` keeps the defaults); the choice is in `config`.

`--impl reference` times the FP64 oracle (the only reference there is: the
paper has no code) on the host on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one per rank (the single-grid step
is not sharded); value = cells x steps of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pf_inputs as I  # noqa: E402

METRIC = "Mcell-steps/s per pf_step"
UNIT = "Mcell-steps/s"
FALLBACK_HBM_GBS = 6800.0


# ---------------------------------------------------------------------------
def workload(name, n=None):
    if name == "osc384":
        p = I.oscillating_drop_384(precision="mixed", n=n or 384)
        desc = (f"3D mode-2 oscillating drop {p['n'][0]}^3 periodic, R=0.25, a=0.05R, "
                "rho ratio 10, mu ratio 10, ACDI + EB, mixed precision")
    elif name == "osc384_fp64":
        p = I.oscillating_drop_384(precision="fp64", n=n or 384)
        desc = f"same drop {p['n'][0]}^3, plain FP64"
    elif name == "drop256":
        p = I.static_drop_256_r1000(precision="mixed")
        desc = "2D static drop 256^2, rho ratio 1000, mu ratio 100, ACDI + EB, mixed"
    elif name in ("batch256", "batch256_fp64"):
        prec = "fp64" if name.endswith("fp64") else "mixed"
        plist = I.batch_manifest(count=256, precision=prec,
                                 poisson_rtol=1e-12 if prec == "fp64" else 1e-10)
        cells = sum(q["n"][0] * q["n"][1] for q in plist)
        desc = (f"256 2D drops, N ~ U{{64..512}} (seed {I.BATCH_SEED}), R in [0.15, 0.3], "
                f"La log-uniform in [1e2, 1e5], rho ratio in {{1, 10, 1000}}, "
                f"static or mode-2, {prec}, {cells} cells in total")
        return plist, desc
    elif name == "osc384_consistent":
        p = I.oscillating_drop_384(precision="mixed", n=n or 384, model="cdi")
        p["momentum"] = "consistent"
        desc = (f"3D mode-2 oscillating drop {p['n'][0]}^3, rho ratio 10, CDI + EB, mixed, "
                "consistent (conservative) momentum transport")
    elif name == "drop256_consistent":
        p = dict(I.static_drop_256_r1000(precision="mixed", model="cdi"), momentum="consistent")
        desc = ("2D static drop 256^2, rho ratio 1000, mu ratio 100, CDI + EB, mixed, "
                "consistent (conservative) momentum transport")
    elif name == "drop64":
        p = I.static_drop_64()
        desc = "2D static drop 64^2, FP64, CDI + EB, La = 12000"
    else:
        raise SystemExit(f"unknown workload {name}")
    return p, desc


def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d and isinstance(d[k], (int, float)):
                return float(d[k]), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def bind_to_gpu_host_cpus(index):
    """Restrict this process to the host CPUs attached to GPU `index` (its PCI
    device's local_cpulist), so that pinned host buffers are allocated in the
    GPU's local memory node; returns the CPU list or None when unknown."""
    import torch

    try:
        pr = torch.cuda.get_device_properties(index)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            text = f.read().strip()
        cpus = set()
        for part in text.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return text
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples go to $PF_CLOCK_DIR (default: the temporary directory)
        d = os.environ.get("PF_CLOCK_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes per cell per launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the 256^3 case of the finest sweep (the TMA-staged
# kernel), mean of the pre- and post-smoothing launches (10.9 and 15.4 B/cell);
# scaled to a launch by the cell count. Valid for the kernel as profiled; None
# for every other class.
# mean of the zero-start and post-smoothing launches of the library's default
# finest sweep (TMA staging, sweep_tile 0)
NCU_TRAFFIC_PER_CELL = {"mg_gs_level0": 13.09}
NCU_TRAFFIC_NOTE = ("ncu DRAM bytes per cell of a 256^3 capture scaled to this grid by the cell "
                    "count: a lower bound (at 256^3 part of the reads hit the 129 MB L2)")


def deal(items, rank, world):
    """The instances of rank `rank` of `world`: item i goes to rank i mod world
    (every item to exactly one rank; no data-path exchange)."""
    return list(items)[rank::world]


def job_time(seconds, dist=None, device=None):
    """The job's time: the slowest rank's (a MAX all-reduce when distributed)."""
    if dist is None:
        return float(seconds)
    import torch

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algo_bytes_per_cell(cls, dim, w, fused_stage=False):
    d = dim
    # the 3D float32 path forms the CG operator's and the finest restriction's
    # coefficients from the cell densities (one array) instead of d face arrays
    ncoef = 1 if (dim == 3 and w == 4) else d
    table = {
        # one full red-black sweep of the finest level (weights from phi), mean
        # of the pre-smoothing sweep (zero start: read f, phi; write x) and the
        # post-smoothing sweep (read x, f, phi, and q for the fused dots; write x)
        "mg_gs_level0": 0.5 * (3 * w + 5 * w),
        # p = z + beta p, q = A p: read z, p and the coefficients (cell densities
        # or d face arrays); write p, q
        "cg_dir_spmv": (2 + ncoef + 2) * w,
        # e += a p, r -= a q: read e, p, r, q; write e, r
        "cg_update": 6 * w,
        # r.z, z.q: read z, r, q
        "cg_dots": 3 * w,
        # r = f - A x to float64 accuracy: read x and b (float64, or double-float
        # pairs on the mixed path), the d face arrays; write r
        "ir_residual_f64": 16 + d * w + w,
        # stage kernel: read phi_s, u_s, phi^n, u^n, normals, mu, accumulators;
        # write phi, u*, accumulators (stages 1-2; the first and last move less)
        # fused stage (no cell pass): read phi_s, u_s, phi^n, u^n, accumulators;
        # write phi, u*, accumulators (stages 1-2)
        "stage": ((1 + d + 1 + d + 1 + d) * w + (1 + d + 1 + d) * w if fused_stage
                  else (1 + d + 1 + d + d + 1 + 1 + d) * w + (1 + d + 1 + d) * w),
        "cell_pass": w + (d + 1) * w,
        "correct": d * w + 8 + d * w + d * w,
        "divergence": d * w + 8,
        "mg_restrict": (2 + ncoef) * w + w / (2 ** d),
        "mg_prolong": 2 * w + w / (2 ** d),
        # float32 face coefficients (and cell densities) from phi
        "beta0_f64": w + d * w + w,
        # x += e with x a double-float (float64 path: float64) pressure
        "ir_addcorr": 2 * (8 if w == 4 else w) + w,
        "gamma": d * w,
    }
    return table.get(cls)


# kernel classes that work on the finest grid (one launch covers every cell);
# the coarse multigrid classes run on levels of 1/2^d, 1/4^d, ... the cells
FINEST_CLASSES = ("mg_gs_level0", "cg_dir_spmv", "cg_update", "ir_residual_f64", "stage",
                  "cell_pass", "correct", "divergence", "beta0_f64", "ir_addcorr", "gamma")


def mg_levels(n, dim, coarse_cells=4096):
    """Cells of the tiled multigrid levels (those below the single-CTA coarse
    solve), finest first, by the library's rule: a level has a coarser one
    while every axis is even and at least 4; the first level of at most
    `coarse_cells` cells (else the coarsest) starts the single-CTA solve."""
    dims = list(n[:dim])
    allc = []
    while True:
        c = 1
        for v in dims:
            c *= v
        allc.append(c)
        if not all(v % 2 == 0 and v >= 4 for v in dims):
            break
        dims = [v // 2 for v in dims]
    first_coarse = next((i for i, c in enumerate(allc) if c <= coarse_cells), len(allc) - 1)
    return allc[:first_coarse]


DENSITY_LEVELS = 1   # coarse levels rediscretised from cell densities (3D float32 path)


def coarse_class_bytes(levels, dim, w, pre=1, post=1):
    """Algorithmic bytes of one V-cycle, per multigrid class that spans several
    levels: the coarse tiled levels' sweeps (pre-smoothing from zero: f and
    the coefficients -> x; further sweeps x, f and the coefficients -> x), the
    restrictions (x, f and the coefficients, plus the coarse write) and the
    prolongations (read-add-write of the fine correction plus the coarse read),
    each level's cells times its bytes per cell. The coefficients are one
    array of cell densities on the 3D float32 path's finest level and its
    first DENSITY_LEVELS coarse levels, else the d face arrays."""
    def ncoef(i):
        return 1 if (dim == 3 and w == 4 and i <= DENSITY_LEVELS) else dim
    frac = 1.0 / 2 ** dim
    gs = sum(c * ((1 + ncoef(i) + 1) * w + (pre - 1 + post) * (1 + 1 + ncoef(i) + 1) * w)
             for i, c in enumerate(levels) if i >= 1)
    rs = sum(c * (((2 + ncoef(i)) * w) + w * frac) for i, c in enumerate(levels))
    pr = sum(c * (2 * w + w * frac) for c in levels)
    return {"mg_gs_coarse_levels": gs, "mg_restrict": rs, "mg_prolong": pr}


def step_roofline(prof, ncell, dim, w, ms_total, ms_host, peak, levels=None, vcycles=None,
                  pre=1, post=1):
    """Compulsory bytes of the kernel classes over the whole timed region,
    divided by the headline time: the finest-grid classes (algorithmic bytes
    per cell x cells x launches) and, given the multigrid levels and the
    number of V-cycles, the classes that span the tiled levels (their bytes
    per V-cycle x V-cycles). The single-CTA coarse solve and the once-per-solve
    coarsening of the coefficients are left out, so the figure is still a
    lower bound. Also the share of the host-driven step time these classes
    take."""
    tot_b, tot_ms = 0.0, 0.0
    classes = []
    for cls in FINEST_CLASSES:
        if cls in prof and prof[cls][0] > 0:
            bpc = algo_bytes_per_cell(cls, dim, w, fused_stage="cell_pass" not in prof)
            tot_b += bpc * ncell * prof[cls][0]
            tot_ms += prof[cls][1]
            classes.append(cls)
    if levels and vcycles:
        for cls, b in coarse_class_bytes(levels, dim, w, pre, post).items():
            if cls in prof and prof[cls][0] > 0 and b > 0:
                tot_b += b * vcycles
                tot_ms += prof[cls][1]
                classes.append(cls)
    if tot_b == 0.0 or ms_total <= 0:
        return None
    achieved = tot_b / (ms_total / 1e3) / 1e9
    return {"bound": "hbm", "bytes": tot_b, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "classes": classes,
            "their_time_share": tot_ms / ms_host if ms_host > 0 else None,
            "their_bandwidth_gbs": tot_b / (tot_ms / 1e3) / 1e9 if tot_ms > 0 else None}


def cpu_sample_rate(p, steps=2, n=16):
    """The oracle (as it stands) on a bounded sample: `steps` RK4 steps of the same
    drop at n^d cells. Returns (Mcell-steps/s, cores, description)."""
    from oracle import pf_oracle as O

    q = dict(p)
    q["n"] = (n, n, n if p["dim"] == 3 else 1)
    q["eps"] = None
    q["dt"] = None
    q["precision"] = "fp64"
    q = I.finalize(q)
    po = O.params_from(q)
    st = O.initial_state(po)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = O.step(st, po)
    dt = time.perf_counter() - t0
    cells = n ** p["dim"]
    # numpy elementwise stencils and SuperLU run on one core
    cores = 1
    desc = (f"{steps} RK4 steps of the same drop at {n}^{p['dim']} (float64 numpy oracle with "
            f"a sparse direct pressure solve; the full {p['n'][0]}^{p['dim']} grid is out of "
            f"reach of the oracle)")
    return cells * steps / dt / 1e6, cores, desc


def cpu_batch_rate(plist, steps=1, max_n=96):
    """The oracle on the batch's small instances (n <= max_n, at their own
    sizes and parameters), one instance per task on a spawned pool over the
    host cores: cells x steps / wall time of the pool (started and warmed
    before the clock starts). Returns (Mcell-steps/s, cores, description)."""
    import multiprocessing as mp

    from oracle import pf_oracle as O

    sample = [p for p in plist if p["n"][0] <= max_n]
    cores = max(1, min(len(sample), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(O.timed_run, [(None, 0)] * cores)
        t0 = time.perf_counter()
        res = pool.map(O.timed_run, [(p, steps) for p in sample], chunksize=1)
        wall = time.perf_counter() - t0
    cells = sum(r[0] for r in res)
    desc = (f"{steps} step(s) of each of the {len(sample)} instances with N <= {max_n} "
            f"(float64 numpy oracle, sparse direct pressure solves), one instance per task "
            f"on {cores} spawned processes")
    return cells / wall / 1e6, cores, desc


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    p, desc = workload(args.workload, args.n)
    vals = []
    for _ in range(args.warmup):
        cpu_sample_rate(p, steps=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, sdesc = cpu_sample_rate(p, steps=1)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall / max(args.steps, 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "sample": sdesc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sdesc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world, local_rank):
    """Throughput of the batched executor on the seeded 256-drop manifest (host
    wall clock bracketed by device synchronisation: the instances run on their
    own streams). Under torchrun the instances are dealt to the ranks
    (instance i to rank i mod N, no collective on the data path); the job's
    time is the slowest rank's."""
    import torch

    import paper_2205_05835_gb300 as pf

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    plist, desc = workload(args.workload)
    total_cells = sum(int(np.prod([c for c in p["n"]])) for p in plist)
    mine = deal(plist, rank, world)
    if args.graph:
        mine = [dict(p, use_graph=1) for p in mine]
    tuned = None
    if args.autotune:
        # multigrid launch shape per grid size, tuned on the size's hardest
        # instance (largest density ratio) before the timed region
        from paper_2205_05835_gb300 import autotune

        tuned = {}
        t_tune = time.perf_counter()
        for n in sorted({p["n"][0] for p in mine}):
            same = [p for p in mine if p["n"][0] == n]
            rep = max(same, key=lambda q: q["rho_in"] / q["rho_out"])
            tuned[n] = autotune.tune(rep)["choice"]
        mine = [autotune.apply(p, {"choice": tuned[p["n"][0]]}) for p in mine]
        t_tune = time.perf_counter() - t_tune
    bat = pf.Batch(mine, nthreads=args.threads)
    bat.step(args.warmup)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    barrier()
    clocks.start()
    t0 = time.perf_counter()
    bat.step(args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier()
    clk = clocks.stop()
    bat.close()
    if dist is not None:
        wall = job_time(wall, dist, "cuda")
        dist.destroy_process_group()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sdesc = cpu_batch_rate(plist)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sdesc}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": total_cells * args.steps / wall / 1e6, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f64" if "fp64" in args.workload else "f32+f64",
            "data": "synthetic",
            "config": {"workload": desc, "cells": total_cells,
                       "threads": 1 if args.graph else args.threads,
                       "execution": "one captured CUDA graph per instance step, device-driven "
                                    "solver loops" if args.graph else "host-driven, thread pool",
                       "parallelism": f"instances dealt to {world} ranks" if world > 1
                       else "single",
                       "timing": "host wall clock between device synchronisations, max over ranks",
                       "autotune": ({"choices": {str(k): v for k, v in tuned.items()},
                                     "tuning_s": t_tune} if tuned is not None else None)},
            "cpu_baseline": cpu, "clocks": clk}), flush=True)


def fp64_baseline(pf, torch, p, stream, local_rank, graph, steps=3):
    """The plain float64 GPU path on the same drop at the float64 accuracy
    (poisson_rtol 1e-12): one untimed step (graph capture), then `steps` timed
    steps with CUDA events and sampled clocks. Beside it, the mixed path runs
    the same 1 + steps steps from the same initial phase field (its float32
    values), and the per-field max-norm distance of the two results, relative
    to the float64 field's maximum, is reported."""
    use_graph = 1 if graph else 0
    with torch.cuda.stream(stream):
        mix = pf.Simulation(dict(p, use_graph=use_graph), stream=stream)
    phi0 = mix.field("phi")
    mix.step(1 + steps)
    names = ("phi", "u", "v", "w", "p") if int(p["dim"]) == 3 else ("phi", "u", "v", "p")
    mfields = {c: mix.field(c) for c in names}
    mix.close()
    del mix
    torch.cuda.empty_cache()
    q = dict(p, precision="fp64", poisson_rtol=1e-12, use_graph=use_graph)
    with torch.cuda.stream(stream):
        sim = pf.Simulation(q, phi0=phi0, stream=stream)
    sim.step(1)
    clocks = ClockSampler(local_rank)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    diag = sim.diagnostics()
    dist = {}
    for c, mv in mfields.items():
        fv = sim.field(c)
        dist[c] = float(np.max(np.abs(mv - fv)) / max(float(np.max(np.abs(fv))), 1e-300))
    ncell = sim.ncell
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return {"value": ncell * steps / (ms / 1e3) / 1e6, "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps, "poisson_rtol": 1e-12,
            "poisson_relres_last": diag["poisson_relres"], "dtype": "f64",
            "execution": "one replayed CUDA graph per step" if graph else "host-driven",
            "clocks": clk,
            "mixed_vs_fp64_after_steps": 1 + steps,
            "mixed_vs_fp64_rel_maxnorm": dist}


def run_ours(args, rank, world, local_rank):
    """Timed steps of one grid per rank. With graph mode (the default) the
    headline number comes from replayed step graphs; the per-kernel CUDA-event
    timings behind the roofline and the kernel shares come from a host-driven
    pass of the same steps from the same initial state (a graph replay cannot
    bracket single kernels with events; the kernels are the same)."""
    import torch

    import paper_2205_05835_gb300 as pf

    torch.cuda.set_device(local_rank)
    host_cpus = bind_to_gpu_host_cpus(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    p, desc = workload(args.workload, args.n)
    if args.inner_tol is not None:
        p["inner_tol"] = args.inner_tol
    if args.mg_sweeps is not None:
        p["mg_pre"] = p["mg_post"] = args.mg_sweeps
    if args.sweep_staging is not None:
        p["sweep_staging"] = args.sweep_staging
    if args.sweep_tile is not None:
        p["sweep_tile"] = args.sweep_tile
    tuned = None
    if args.autotune and args.mg_sweeps is None:
        # multigrid launch shape tuned on this grid before the timed region
        from paper_2205_05835_gb300 import autotune

        t_tune = time.perf_counter()
        r = autotune.tune(dict(p, use_graph=1 if args.graph else 0), steps=2, warm=1)
        p = autotune.apply(p, r)
        tuned = {"choice": r["choice"], "ms_per_step": r["ms_per_step"],
                 "tuning_s": time.perf_counter() - t_tune}
    stream = torch.cuda.Stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(sim, profile):
        for _ in range(args.warmup):
            sim.step(1)
        if profile:
            pf.pf_profile_read(sim.ctx, reset=True)
            pf.pf_profile_enable(sim.ctx, True)
        clocks = ClockSampler(local_rank)
        barrier()
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        barrier()
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1)
        prof = None
        if profile:
            prof = pf.pf_profile_read(sim.ctx, reset=True)
            pf.pf_profile_enable(sim.ctx, False)
        return ms, clk, prof, sim.diagnostics()

    # host-driven pass: per-kernel CUDA events (the whole measurement when
    # graph mode is off)
    with torch.cuda.stream(stream):
        sim = pf.Simulation(p, stream=stream)
    ncell = sim.ncell
    ms_h, clk, prof, diag = timed(sim, True)
    ms = ms_h
    if args.graph:
        sim.close()
        del sim
        torch.cuda.empty_cache()
        with torch.cuda.stream(stream):
            sim = pf.Simulation(dict(p, use_graph=1), stream=stream)
        ms, clk, _, diag = timed(sim, False)
    ms = job_time(ms, dist, "cuda")
    ms_step = ms / args.steps
    value = ncell * world * args.steps / (ms / 1e3) / 1e6
    launches = int(sum(v[0] for v in prof.values()))

    # dominant kernel class and its roofline (host-driven pass)
    w = 4 if p["precision"] == "mixed" else 8
    ranked = sorted(((v[1], k, v[0]) for k, v in prof.items() if v[0] > 0), reverse=True)
    dom_ms, dom, dom_n = ranked[0] if ranked else (0.0, None, 0)
    peak, peak_kind = measured_hbm()
    bpc = algo_bytes_per_cell(dom, p["dim"], w, fused_stage="cell_pass" not in prof)
    roof = None
    if bpc is not None and dom_n > 0:
        avg_s = dom_ms / dom_n / 1e3
        achieved = bpc * ncell / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (NCU_TRAFFIC_PER_CELL[dom] * ncell
                            if dom in NCU_TRAFFIC_PER_CELL and p["dim"] == 3
                            and p.get("precision") == "mixed"
                            and not p.get("sweep_tile") and not p.get("sweep_staging")
                            else None),
                "traffic_note": (NCU_TRAFFIC_NOTE if dom in NCU_TRAFFIC_PER_CELL else None),
                "algo_bytes_per_launch": bpc * ncell,
                "avg_launch_us": avg_s * 1e6,
                "share_of_step": dom_ms / ms_h if ms_h > 0 else None,
                "timed_in": ("host-driven pass of the same steps (CUDA events around "
                             "each launch)" if args.graph else "the timed steps")}
    pre = int(p.get("mg_pre", 0) or 1)
    post = int(p.get("mg_post", 0) or 1)
    levels = mg_levels(p["n"], p["dim"], int(p.get("mg_coarse_cells", 0) or 4096))
    vcycles = prof.get("mg_coarse_vcycle", (0, 0.0))[0] if "mg_coarse_vcycle" in prof else 0
    step_roof = step_roofline(prof, ncell, p["dim"], w, ms, ms_h, peak, levels=levels,
                              vcycles=vcycles, pre=pre, post=post)

    # end to end through the C ABI: state from / to pinned host memory every step
    e2e = None
    if not args.no_e2e:
        nb = sim.state_bytes()
        h_in = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        h_out = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        pf.pf_get_state(sim.ctx, h_in.data_ptr())
        e2e_steps = max(1, min(args.steps, 5))
        barrier()
        t_h2d = t_step = t_d2h = 0.0
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ta = time.perf_counter()
            pf.pf_set_state(sim.ctx, h_in.data_ptr())      # synchronises
            tb = time.perf_counter()
            sim.step(1)
            pf.pf_sync(sim.ctx)
            tc = time.perf_counter()
            pf.pf_get_state(sim.ctx, h_out.data_ptr())     # synchronises
            td = time.perf_counter()
            t_h2d += tb - ta
            t_step += tc - tb
            t_d2h += td - tc
        barrier()
        et = time.perf_counter() - t0
        e2e = {"value": ncell * world * e2e_steps / et / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb, "steps": e2e_steps,
               "host_cpus": host_cpus,
               "ms_per_step": {"h2d": 1e3 * t_h2d / e2e_steps, "step": 1e3 * t_step / e2e_steps,
                               "d2h": 1e3 * t_d2h / e2e_steps}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sdesc = cpu_sample_rate(p, steps=6)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sdesc}

    fp64 = None
    if rank == 0 and world == 1 and args.fp64 and p["precision"] == "mixed":
        sim.close()
        del sim
        torch.cuda.empty_cache()
        fp64 = fp64_baseline(pf, torch, p, stream, local_rank, args.graph)
        sim = None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if p["precision"] == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": desc, "cells": ncell, "dt": p["dt"],
                       "poisson_rtol": p["poisson_rtol"],
                       "l2": "state > L2 (no flush needed)",
                       "execution": ("one replayed CUDA graph per step (device-driven "
                                     "solver loops)" if args.graph else "host-driven"),
                       "parallelism": "replicas" if world > 1 else "single",
                       "autotune": tuned},
            "roofline": roof, "step_roofline": step_roof, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": launches,
            "gpu_launches_counted_in": ("host-driven pass of the same steps (a replay "
                                        "adds early-exit launches of the unrolled CG "
                                        "pair and the loop-condition kernels)"
                                        if args.graph else "the timed steps"),
            "ms_per_step_host_driven": ms_h / args.steps,
            "poisson_iters_last": diag["poisson_iters"],
            "poisson_iters_max": diag["poisson_iters_max"],
            "poisson_relres_last": diag["poisson_relres"],
            "kernel_ms": {k: round(v[1], 3) for k, v in prof.items() if v[0] > 0},
            "kernel_launches": {k: v[0] for k, v in prof.items() if v[0] > 0},
            "fp64_baseline": fp64,
        }
        print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="osc384")
    ap.add_argument("--n", type=int, default=None, help="override the grid size (testing)")
    ap.add_argument("--threads", type=int, default=16, help="host threads (batch workload)")
    ap.add_argument("--inner-tol", type=float, default=None,
                    help="relative reduction of each float32 inner solve (mixed path)")
    ap.add_argument("--mg-sweeps", type=int, default=None,
                    help="pre- and post-smoothing sweeps per V-cycle (tuning; default 1)")
    ap.add_argument("--sweep-staging", type=int, default=None,
                    help="finest-level sweeps: 0 TMA-staged (the library's default), 1 cp.async")
    ap.add_argument("--sweep-tile", type=int, default=None,
                    help="TMA-staged sweeps' tile shape (pf_params.sweep_tile, 0 .. 4)")
    ap.add_argument("--graph", type=int, default=1,
                    help="1 (default): replay one captured CUDA graph per step (use_graph); "
                         "0: host-driven solver loops")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1 (default): tune the multigrid launch shape (per grid size for the "
                         "batch) before the timed region")
    ap.add_argument("--fp64", type=int, default=1,
                    help="1 (default, mixed workloads, one GPU): also time the plain FP64 "
                         "GPU path on the same grid and report the mixed result's distance")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload.startswith("batch"):
        run_batch(args, rank, world, local_rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
