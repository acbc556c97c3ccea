"""Whole steps of the benchmarked 3D mixed-precision path against the FP64 oracle.

3D float32 grids run the column-marching stage, cell-pass, divergence and
correction kernels, the one-pass tiled red-black sweeps, the register-marching
direction / operator product and the double-float outer residual. Here they
run together, as whole RK4 steps, on grids that span several 32 x 8 tiles
with a ragged tail in x, and the result is compared with the float64 oracle
element by element on the same float32-rounded initial phase field.

Stated per-field bounds of the mixed path (max-norm, relative to the field's
maximum), the same as for the 2D mixed step: phi < 1e-5, u < 2e-3, p < 1e-4;
mass conserved to 1e-6 relative per step (phi is stored in float32).

The second test runs the 384^3 drop itself for 50 steps in mixed precision
and in plain float64 on the GPU and records how the per-field distance and
the mass drift grow with the step count.
"""
import numpy as np
import pytest

import pf_inputs as I
from oracle import pf_oracle as O

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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


@pytest.mark.parametrize("n,model", [((40, 24, 16), "cdi"), ((32, 16, 16), "cdi"),
                                     ((40, 24, 16), "acdi")])
def test_mixed_3d_steps_match_oracle(pf, n, model):
    steps = 3
    p = I.small_case(dim=3, n=n[0], precision="mixed", poisson_rtol=1e-10, model=model)
    p["n"] = n
    p = I.finalize(p)
    po = O.params_from(p)
    phi0 = O.initial_phi(po).astype(np.float32).astype(np.float64)
    sim = pf.Simulation(p, phi0=phi0)
    m0 = sim.diagnostics()["mass"]
    sim.step(steps)
    d = sim.diagnostics()
    st = O.run(dict(po, precision="fp64"), steps=steps, phi0=phi0)
    errs = {"phi": rel(sim.field("phi"), st.phi), "p": rel(sim.field("p"), st.p)}
    for c, ref in zip("uvw", st.u):
        errs[c] = rel(sim.field(c), ref)
    print("mixed 3D", model, n, errs)
    sim.close()
    assert errs["phi"] < 1e-5, errs
    assert max(errs["u"], errs["v"], errs["w"]) < 2e-3, errs
    assert errs["p"] < 1e-4, errs
    assert abs(d["mass"] / m0 - 1.0) < steps * 1e-6
    od = O.diagnostics(st, po)
    assert abs(d["ke"] - od["ke"]) <= 4e-3 * od["ke"]
    assert d["poisson_relres"] <= p["poisson_rtol"]


def test_mixed_384_fifty_steps_against_fp64(pf):
    """The benchmarked drop, mixed against plain float64 on the GPU over 50
    steps (a tenth of its 500): per-field distance within the one-step bounds
    times the step count's square root, and mass drift within 1e-6 per step."""
    p = I.oscillating_drop_384(precision="mixed")
    po = O.params_from(p)
    phi0 = O.initial_phi(po).astype(np.float32).astype(np.float64)
    mix = pf.Simulation(p, phi0=phi0)
    f64 = pf.Simulation(dict(p, precision="fp64", poisson_rtol=1e-12), phi0=phi0)
    m0 = f64.diagnostics()["mass"]
    done = 0
    rows = []
    for target in (1, 10, 25, 50):
        mix.step(target - done)
        f64.step(target - done)
        done = target
        e = {c: rel(mix.field(c), f64.field(c)) for c in ("phi", "u", "v", "w", "p")}
        dm = mix.diagnostics()["mass"] / m0 - 1.0
        d64 = f64.diagnostics()["mass"] / m0 - 1.0
        rows.append((target, e, dm, d64))
        print("384^3 step", target, e, "mass drift mixed", dm, "fp64", d64)
    mix.close()
    f64.close()
    for k, e, dm, d64 in rows:
        s = np.sqrt(k)
        assert e["phi"] < 1e-6 * s * 2, (k, e)
        assert max(e["u"], e["v"], e["w"]) < 1e-3 * s, (k, e)
        assert e["p"] < 1e-4 * s, (k, e)
        assert abs(dm) < 1e-6 * k, (k, dm)
        assert abs(d64) < 1e-13 * k, (k, d64)
