"""Graph mode (use_graph = 1): pf_step replays one captured CUDA graph per step,
the pressure solves' CG and refinement loops as device-driven WHILE nodes.
It runs the same kernels in the same order with the same early exits as the
host-driven loops, so every field must agree bit for bit."""
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


CASES = [
    dict(dim=2, n=48, precision="fp64", scheme="rk4", poisson_rtol=1e-12),
    dict(dim=2, n=64, precision="mixed", scheme="rk4", rho_in=1000.0, poisson_rtol=1e-10),
    dict(dim=2, n=40, precision="fp64", scheme="fe", force="lcsf", poisson_rtol=1e-12),
    dict(dim=3, n=32, precision="mixed", scheme="rk4", poisson_rtol=1e-10),
    dict(dim=3, n=16, precision="fp64", scheme="rk4", model="sb", poisson_rtol=1e-12),
]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: f"{k['dim']}d-{k['n']}-{k['precision']}-{k['scheme']}")
def test_graph_steps_equal_host_steps(pf, kw):
    p = I.small_case(**kw)
    a = pf.Simulation(p)
    b = pf.Simulation(dict(p, use_graph=1))
    a.step(5)
    b.step(2)    # capture, two replays
    b.step(3)    # three more replays
    names = ("phi", "u", "v", "w", "p") if kw["dim"] == 3 else ("phi", "u", "v", "p")
    for name in names:
        np.testing.assert_array_equal(a.field(name), b.field(name), err_msg=name)
    da, db = a.diagnostics(), b.diagnostics()
    assert da["step"] == db["step"] == 5
    assert da["poisson_iters"] == db["poisson_iters"]
    assert da["gamma"] == db["gamma"]
    a.close()
    b.close()


def test_graph_batch_equals_individual_contexts(pf):
    plist = []
    for n, ratio, prec, mode in [(48, 10.0, "fp64", 2), (64, 1000.0, "mixed", 0),
                                 (32, 1.0, "fp64", 2), (80, 10.0, "mixed", 2)]:
        plist.append(I.small_case(dim=2, n=n, rho_in=ratio, rho_out=1.0, precision=prec,
                                  pert_mode=mode, pert_amp=0.05 if mode else 0.0,
                                  poisson_rtol=1e-11, use_graph=1))
    bat = pf.Batch(plist)
    bat.step(2)
    bat.step_each([1, 0, 2, 1])
    counts = [3, 2, 4, 3]
    for i, p in enumerate(plist):
        sim = pf.Simulation(dict(p, use_graph=0))
        sim.step(counts[i])
        assert bat.diagnostics(i)["step"] == counts[i]
        for name in ("phi", "u", "v", "p"):
            np.testing.assert_array_equal(bat.field(i, name), sim.field(name), err_msg=name)
        sim.close()
    bat.close()


def test_graph_mode_reports_iteration_cap(pf):
    """A solve stopped by poisson_maxit inside a replay is reported after it."""
    p = I.small_case(dim=2, n=32, poisson_rtol=1e-14, poisson_maxit=2, use_graph=1)
    sim = pf.Simulation(p)
    with pytest.raises(pf.PFError) as e:
        sim.step(3)
    assert e.value.status == pf.B.PF_ERR_NOT_CONVERGED
    sim.close()
