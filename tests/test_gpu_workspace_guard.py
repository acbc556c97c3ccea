"""The context stays inside the workspace that pf_workspace_size sizes.

The workspace is carved twice from the same parameters: once from a null base
to count the bytes, once for real. A buffer whose presence the real pass
decides differently from the counting pass would be written past the end of
the caller's allocation. Here every context gets its exact byte count followed
by a guard region with a fixed pattern; after steps and a pressure solve the
guard must be untouched.
"""
import numpy as np
import pytest

import pf_inputs as I
from oracle import pf_oracle as O

pytestmark = pytest.mark.gpu

GUARD = 1 << 20
PATTERN = 0x5A


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2205_05835_gb300 as pf

    return pf, torch


CASES = [
    (3, (96, 48, 32), "mixed", {}),
    (3, (96, 48, 32), "mixed", {"sweep_staging": 1}),
    (3, (96, 48, 32), "mixed", {"sweep_tile": 2}),
    (3, (64, 64, 64), "mixed", {"mg_coarse_cells": 1024}),
    (3, (32, 32, 32), "fp64", {}),
    (2, (64, 64, 1), "mixed", {}),
    (2, (128, 128, 1), "fp64", {"mg_pre": 2, "mg_post": 2}),
]


@pytest.mark.parametrize("dim,n,precision,knobs", CASES)
def test_context_writes_only_its_workspace(env, dim, n, precision, knobs):
    pf, torch = env
    p = I.small_case(dim=dim, n=n[0], rho_in=10.0, rho_out=1.0, precision=precision,
                     poisson_rtol=1e-10)
    p["n"] = n if dim == 3 else (n[0], n[1])
    p = dict(I.finalize(p), **knobs)
    prm = pf.make_params(p)
    nbytes = pf.pf_workspace_size(prm)
    dev = torch.device("cuda", 0)
    buf = torch.full((nbytes + 256 + GUARD,), PATTERN, dtype=torch.uint8, device=dev)
    base = (buf.data_ptr() + 255) // 256 * 256
    off = base - buf.data_ptr()
    stream = torch.cuda.current_stream(dev)
    ctx = pf.pf_init(prm, base, nbytes, None, stream.cuda_stream)
    try:
        pf.pf_step(ctx, 2)
        g = O.Grid(dim, p["n"], p["L"])
        rhs = I.noise(g.shape, 5) - 0.5
        rhs -= rhs.mean()
        x = np.zeros(rhs.size)
        st, it, rel = pf.pf_poisson_solve(ctx, np.ascontiguousarray(rhs.ravel()).ctypes.data,
                                          x.ctypes.data)
        assert st == 0 and rel <= 1e-10
    finally:
        pf.pf_destroy(ctx)
    torch.cuda.synchronize()
    tail = buf[off + nbytes:].cpu().numpy()
    assert tail.size >= GUARD
    bad = np.flatnonzero(tail != PATTERN)
    assert bad.size == 0, f"{bad.size} guard bytes overwritten, first at +{int(bad[0])}"
