"""Failure detection of the TMA-staged sweep's bounded waits, without a GPU fault.

Every mbarrier wait of the finest-level sweep gives up after about one second
of the global timer, latches PF_ERR_TIMEOUT in the solve's scalars, lets its
copies in flight land (bounded again) and returns, so the context stays usable.
With PF_TEST_SWEEP_STALL set when a context is created, one interior CTA of its
sweeps expects 16 bytes more than a plane brings: that barrier phase never
completes (a flag that nothing sets), the copies themselves all land, and the
waits run out. The solve reports the timeout within seconds; the same context
then still answers, and a context created without the variable solves to the
tolerance.
"""
import time

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


def test_sweep_wait_timeout_is_reported_and_context_stays_usable(pf, monkeypatch):
    n = (96, 32, 16)
    p = I.small_case(dim=3, n=n[0], rho_in=10.0, rho_out=1.0, precision="mixed",
                     poisson_rtol=1e-10, poisson_maxit=200)
    p["n"] = n
    po = O.params_from(p)
    g = O.Grid(3, n, p["L"])
    phi = O.initial_phi(po)
    rhs = I.noise(g.shape, 29) - 0.5
    rhs -= rhs.mean()
    monkeypatch.setenv("PF_TEST_SWEEP_STALL", "1")
    sim = pf.Simulation(p, phi0=phi)
    monkeypatch.delenv("PF_TEST_SWEEP_STALL")
    t0 = time.time()
    with pytest.raises(pf.PFError) as e:
        sim.poisson_solve(rhs)
    took = time.time() - t0
    assert e.value.status == pf.B.PF_ERR_TIMEOUT, e.value
    assert "bounded wait" in str(e.value)
    assert 0.5 < took < 30.0, took
    # the context still answers (diagnostics synchronise and reduce)
    d = sim.diagnostics()
    assert np.isfinite(d["mass"]) and d["mass"] > 0
    sim.close()
    sim2 = pf.Simulation(p, phi0=phi)
    x2, it2, rel2, st2 = sim2.poisson_solve(rhs)
    sim2.close()
    assert st2 == 0 and rel2 <= 1e-10
