"""The multigrid launch-shape autotuner on the GPU: every candidate gives the
oracle's answer (the knobs change the preconditioner only), and tune() picks
one of the candidates, caching it per signature."""
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


@pytest.mark.parametrize("dim,n,cells,sweeps", [(2, 80, 64, 1), (2, 80, 16384, 1),
                                                (2, 48, 4096, 2), (3, 24, 64, 1),
                                                (3, 24, 16384, 2)])
def test_every_launch_shape_gives_the_oracle_answer(pf, dim, n, cells, sweeps):
    p = I.small_case(dim=dim, n=n, poisson_rtol=1e-13, poisson_maxit=400,
                     mg_coarse_cells=cells, mg_pre=sweeps, mg_post=sweeps)
    po = O.params_from(p)
    sim = pf.Simulation(p)
    sim.step(2)
    st = O.run(po, steps=2)
    assert rel(sim.field("phi"), st.phi) < 1e-10
    for d in range(dim):
        assert rel(sim.field("uvw"[d]), st.u[d]) < 1e-10
    sim.close()


def test_tune_picks_a_candidate_and_caches(pf):
    from paper_2205_05835_gb300 import autotune

    p = I.small_case(dim=2, n=128, precision="mixed", poisson_rtol=1e-10, use_graph=1)
    r = autotune.tune(p, steps=2, warm=1, tune_inner=True)
    shape = {k: v for k, v in r["choice"].items() if k != "inner_tol"}
    assert shape in list(autotune.CANDIDATES) and not r["cached"]
    assert r["choice"].get("inner_tol", 1e-6) in autotune.INNER_TOLS
    assert len(r["ms_per_step"]) == len(autotune.CANDIDATES) + len(autotune.INNER_TOLS) - 1
    assert all(v > 0 for v in r["ms_per_step"].values())
    assert autotune.tune(p, tune_inner=True)["cached"]
    sim = pf.Simulation(autotune.apply(p, r))
    sim.step(3)
    assert sim.diagnostics()["poisson_relres"] < 1e-10
    sim.close()


def test_tune_picks_a_sweep_tile_on_a_3d_mixed_grid(pf):
    """3D mixed precision: the tile shape of the TMA-staged finest sweep is tuned
    after the multigrid shape; every tile gives a converged solve."""
    from paper_2205_05835_gb300 import autotune

    p = I.small_case(dim=3, n=64, precision="mixed", poisson_rtol=1e-10)
    cands = autotune.CANDIDATES[:2]
    r = autotune.tune(p, candidates=cands, steps=1, warm=1)
    assert not r["cached"]
    assert len(r["ms_per_step"]) == len(cands) + len(autotune.SWEEP_TILES) - 1
    assert r["choice"].get("sweep_tile", 0) in autotune.SWEEP_TILES
    for tile in autotune.SWEEP_TILES:
        sim = pf.Simulation(dict(autotune.apply(p, r), sweep_tile=tile))
        sim.step(2)
        assert sim.diagnostics()["poisson_relres"] < 1e-10
        sim.close()
