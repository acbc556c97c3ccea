"""The allocation-free pressure solve (pf_poisson_solve_static).

Some callers cannot allocate device memory: a framework whose memory pool
owns all device memory, or a real-time loop that must not allocate after
start-up. pf_poisson_solve_static serves them with scratch in a fixed array
inside the library. This file checks, through the C ABI, that two calls in a
row give the same solution as the context-based pf_poisson_solve, within the
tolerance the other Poisson tests use, and as the oracle's exact solve; and
that grids beyond the array's capacity are rejected with a clear error. It is
collected last so that a failure here leaves every other test already run; it
passes alone in a fresh process too.
"""
import numpy as np
import pytest

import pf_inputs as I
from oracle import pf_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2205_05835_gb300 as pf

    return pf, torch


def beta_f32(phi, g, p):
    """1 / rho_f evaluated and rounded in float32 from float32 phi, as float64."""
    ph = phi.astype(np.float32)
    c = np.clip(ph, np.float32(0), np.float32(1))
    dr = np.float32(np.float32(p["rho_in"]) - np.float32(p["rho_out"]))
    rho = np.float32(p["rho_out"]) + (dr * c).astype(np.float32)
    return [(np.float32(1) / (np.float32(0.5) * (rho + np.roll(rho, 1, axis=g.axis(d)))))
            .astype(np.float64) for d in range(g.dim)]


@pytest.mark.parametrize("dim,n,precision,tol", [(3, 32, "fp64", 1e-9), (2, 96, "fp64", 1e-9),
                                                  (3, 40, "mixed", 1e-7)])
def test_static_solve_matches_context_solve(env, dim, n, precision, tol):
    pf, torch = env
    p = I.small_case(dim=dim, n=n, rho_in=100.0, rho_out=1.0, precision=precision,
                     poisson_rtol=1e-12, poisson_maxit=300)
    po = O.params_from(p)
    g = O.Grid(dim, p["n"], p["L"])
    phi = O.initial_phi(po)
    rhs = I.noise(g.shape, 21) - 0.5
    rhs -= rhs.mean()
    # the existing entry point (context + caller-allocated workspace)
    sim = pf.Simulation(p, phi0=phi)
    want, it_ref, rel_ref, st_ref = sim.poisson_solve(rhs)
    sim.close()
    assert st_ref == 0
    dev = torch.device("cuda", 0)
    d_phi = torch.as_tensor(phi.ravel()).to(dev)
    d_rhs = torch.as_tensor(rhs.ravel()).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    prm = pf.make_params(p)
    for call in range(2):
        d_x = torch.zeros(phi.size, dtype=torch.float64, device=dev)
        st, it, rel = pf.B.pf_poisson_solve_static(prm, d_phi.data_ptr(), d_rhs.data_ptr(),
                                                   d_x.data_ptr(), stream)
        assert st == 0, pf.pf_last_error(None)
        assert rel <= 1e-12
        got = d_x.cpu().numpy().reshape(g.shape)
        err = np.max(np.abs(got - want)) / np.max(np.abs(want))
        assert err < tol, (call, err)
    # and the oracle's exact solve of the same system (the mixed path's
    # operator has float32-rounded face coefficients of float32 phi)
    beta = O.face_beta(phi, g, po) if precision == "fp64" else beta_f32(phi, g, po)
    exact = O.solve_poisson(beta, rhs, g)
    err = np.max(np.abs(got - exact)) / np.max(np.abs(exact))
    assert err < tol, err


def test_static_solve_rejects_oversized_grids(env):
    pf, torch = env
    p = I.small_case(dim=3, n=128, precision="fp64")
    prm = pf.make_params(p)
    dev = torch.device("cuda", 0)
    buf = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(pf.PFError) as e:
        pf.B.pf_poisson_solve_static(prm, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                     torch.cuda.current_stream(dev).cuda_stream)
    assert e.value.status == pf.B.PF_ERR_INVALID
    assert "static scratch" in pf.pf_last_error(None)
