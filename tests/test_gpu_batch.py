"""Batched execution (pf_batch_*): every instance of a batch of uneven drops
computes exactly what pf_step computes on its own context."""
import numpy as np
import pytest

import pf_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2205_05835_gb300 as pf

    return pf


def instances():
    out = []
    for n, ratio, R, prec, force, mode in [(48, 10.0, 0.25, "fp64", "eb", 2),
                                           (64, 1000.0, 0.2, "mixed", "eb", 0),
                                           (32, 1.0, 0.3, "fp64", "csf", 2),
                                           (80, 10.0, 0.15, "mixed", "lcsf", 2),
                                           (40, 100.0, 0.22, "fp64", "eb", 0)]:
        out.append(I.small_case(dim=2, n=n, rho_in=ratio, rho_out=1.0, R=R, precision=prec,
                                force=force, pert_mode=mode, pert_amp=0.05 if mode else 0.0,
                                poisson_rtol=1e-11))
    return out


def test_batch_equals_individual_contexts(pf):
    plist = instances()
    bat = pf.Batch(plist, nthreads=3)
    bat.step(3)
    for i, p in enumerate(plist):
        sim = pf.Simulation(p)
        sim.step(3)
        for name in ("phi", "u", "v", "p"):
            np.testing.assert_array_equal(bat.field(i, name), sim.field(name))
        assert bat.diagnostics(i)["step"] == 3
        sim.close()
    bat.close()


def test_manifest_batch_runs(pf):
    """The seeded manifest of uneven drops (first 24 instances): finite, CDI mass
    conserved to float64/float32 rounding."""
    plist = I.batch_manifest(count=24, precision="fp64", poisson_rtol=1e-11)
    bat = pf.Batch(plist)
    m0 = [bat.diagnostics(i)["mass"] for i in range(len(bat))]
    bat.step(2)
    for i in range(len(bat)):
        d = bat.diagnostics(i)
        assert np.isfinite(d["ke"]) and abs(d["mass"] - m0[i]) <= 1e-9 * m0[i]
    bat.close()


def test_step_each_matches_individual_step_counts(pf):
    """pf_batch_step_each: instance i advances exactly nsteps[i] steps."""
    plist = instances()[:4]
    counts = [2, 0, 3, 1]
    bat = pf.Batch(plist, nthreads=2)
    bat.step_each(counts)
    for i, p in enumerate(plist):
        sim = pf.Simulation(p)
        if counts[i]:
            sim.step(counts[i])
        assert bat.diagnostics(i)["step"] == counts[i]
        for name in ("phi", "u", "p"):
            np.testing.assert_array_equal(bat.field(i, name), sim.field(name))
        sim.close()
    bat.close()
