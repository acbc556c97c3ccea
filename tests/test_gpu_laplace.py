"""Laplace pressure jump of the static drop at density ratio 1000 (256^2,
viscosity ratio 100, CDI; Section 3.1 setup with the EB, CSF and LCSF forces).

(1) Full-size parity: one float64 step on the GPU against one oracle step on
    the same 256^2 input (every field to 1e-10, the jump to 1e-10). With
    eps = dx the discrete EB jump lies 4.6 % below sigma/R in both: that is the
    discretisation (the oracle pins its second-order convergence in dx/eps to
    the PDE value), not a solver error.
(2) The mixed form's jump against the float64 form's, per force, after 50
    steps: within 0.1 %.
(3) With the interface resolved (eps = 8 dx) the EB jump of both forms lies
    within 0.1 % of the PDE value int 6 sigma phi^2 (1-phi)^2 / (eps r) dr.
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


def drop(force="eb", precision="fp64", eps=None, steps=1):
    p = I.static_drop_256_r1000(force=force, precision=precision)
    if eps is not None:
        p = dict(p, eps=eps, dt=None)
    p = dict(p, steps=steps)
    if precision == "mixed":
        p["poisson_rtol"] = 1e-10
    return I.finalize(p)


@pytest.mark.parametrize("force", ["eb", "csf", "lcsf"])
def test_first_step_parity_full_size(pf, force):
    # the static drop's velocity is the small difference of u* and tau beta G p,
    # so the solve runs one decade below the step's 1e-12 to keep u at 1e-10
    p = dict(drop(force), poisson_rtol=1e-13)
    po = O.params_from(p)
    st0 = O.initial_state(po)
    sim = pf.Simulation(p, phi0=st0.phi)
    st = O.step(st0, po)
    sim.step(1)
    assert rel(sim.field("phi"), st.phi) < 1e-10
    assert rel(sim.field("u"), st.u[0]) < 1e-10
    assert rel(sim.field("v"), st.u[1]) < 1e-10
    assert rel(sim.field("p"), st.p - st.p.mean()) < 1e-10
    dp = sim.diagnostics()["dp_laplace"]
    want = O.diagnostics(st, po)["dp_laplace"]
    assert abs(dp / want - 1.0) < 1e-10, (dp, want)
    if force == "eb":
        # eps = dx: the discrete EB jump, about 4.6 % below sigma / R
        assert -0.05 < dp / 4.0 - 1.0 < -0.04, dp
    sim.close()


@pytest.mark.parametrize("force", ["eb", "csf", "lcsf"])
def test_mixed_jump_within_tenth_percent(pf, force):
    a = pf.Simulation(drop(force, "fp64"))
    b = pf.Simulation(drop(force, "mixed"))
    a.step(50)
    b.step(50)
    da = a.diagnostics()["dp_laplace"]
    db = b.diagnostics()["dp_laplace"]
    assert abs(db / da - 1.0) < 1e-3, (da, db)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resolved_eb_jump_within_tenth_percent_of_pde(pf, precision):
    eps = 8.0 / 256
    sim = pf.Simulation(drop("eb", precision, eps=eps))
    sim.step(1)
    dp = sim.diagnostics()["dp_laplace"]
    want = O.laplace_jump_pde(2, 1.0, 0.25, eps)
    assert abs(dp / want - 1.0) < 1e-3, (dp, want)
    sim.close()
