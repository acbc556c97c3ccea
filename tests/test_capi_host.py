"""The C-ABI library loads, exports every entry point include/pf.h declares,
and its host-side validation works (no GPU needed: no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pf():
    import __graft_entry__ as g

    g.build()
    import paper_2205_05835_gb300 as pf

    return pf


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:pf_status|void|size_t|int|const char\*|pf_ctx\*)\s+(pf_\w+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("pf_init", "pf_step", "pf_project", "pf_diagnostics", "pf_workspace_size",
              "pf_destroy", "pf_last_error", "pf_get_state", "pf_set_state"):
        assert s in syms


def test_library_exports_every_declared_symbol(pf):
    import ctypes

    lib = ctypes.CDLL(pf.B.LIB_PATH)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(declared_symbols()) == set(pf.B.SYMBOLS)


def test_workspace_size_and_validation(pf):
    import pf_inputs as I

    p = pf.make_params(I.static_drop_64())
    n64 = pf.pf_workspace_size(p)
    assert n64 > 64 * 64 * 8 * 10
    p2 = pf.make_params(I.oscillating_drop_384(n=64))
    assert pf.pf_workspace_size(p2) > 64 ** 3 * 4 * 20
    # mixed precision needs fewer bytes than fp64 for the same grid
    pm = pf.make_params(dict(I.oscillating_drop_384(n=64), precision="fp64"))
    assert pf.pf_workspace_size(pm) > pf.pf_workspace_size(p2)
    bad = pf.make_params(I.static_drop_64())
    bad.dim = 4
    with pytest.raises(pf.PFError) as e:
        pf.pf_workspace_size(bad)
    assert e.value.status == pf.B.PF_ERR_INVALID
    bad = pf.make_params(I.static_drop_64())
    bad.n[0] = 2
    with pytest.raises(pf.PFError):
        pf.pf_workspace_size(bad)
    bad = pf.make_params(I.static_drop_64())
    bad.dt = 0.0
    with pytest.raises(pf.PFError):
        pf.pf_workspace_size(bad)
    bad = pf.make_params(I.static_drop_64())
    bad.reserved[0] = 1
    with pytest.raises(pf.PFError):
        pf.pf_workspace_size(bad)
    bad = pf.make_params(I.static_drop_64())
    bad.sweep_staging = 2
    with pytest.raises(pf.PFError):
        pf.pf_workspace_size(bad)
    bad = pf.make_params(I.static_drop_64())
    bad.stage_kernel = 2
    with pytest.raises(pf.PFError):
        pf.pf_workspace_size(bad)
    bad = pf.make_params(I.static_drop_64())
    bad.sweep_tile = 5
    with pytest.raises(pf.PFError):
        pf.pf_workspace_size(bad)


def test_init_rejects_bad_workspace_without_touching_the_gpu(pf):
    import ctypes

    import pf_inputs as I

    p = pf.make_params(I.static_drop_64())
    ctx = ctypes.c_void_p(0)
    st = pf.B.LIB.pf_init(ctypes.byref(p), None, 0, None, None, ctypes.byref(ctx))
    assert st == pf.B.PF_ERR_WORKSPACE
    assert "workspace" in pf.pf_last_error(None)
    st = pf.B.LIB.pf_init(ctypes.byref(p), 0x1001, 1 << 40, None, None, ctypes.byref(ctx))
    assert st == pf.B.PF_ERR_WORKSPACE


def test_batch_workspace_is_the_sum_of_aligned_instances(pf):
    import pf_inputs as I

    man = I.batch_manifest(count=5)
    prms = [pf.make_params(p) for p in man]
    total = pf.pf_batch_workspace_size(prms)
    want = sum((pf.pf_workspace_size(q) + 255) // 256 * 256 for q in prms)
    assert total == want
    bad = [pf.make_params(p) for p in man]
    bad[3].dim = 5
    with pytest.raises(pf.PFError) as e:
        pf.pf_batch_workspace_size(bad)
    assert "instance 3" in str(e.value)


def test_batch_manifest_is_seeded_and_in_range():
    import pf_inputs as I

    a = I.batch_manifest(count=256)
    b = I.batch_manifest(count=256)
    assert [p["n"] for p in a] == [p["n"] for p in b]
    ns = [p["n"][0] for p in a]
    assert min(ns) >= 64 and max(ns) <= 512 and all(n % 16 == 0 for n in ns)
    assert all(0.15 <= p["R"] <= 0.3 for p in a)
    assert {p["rho_in"] / p["rho_out"] for p in a} <= {1.0, 10.0, 1000.0}
    cells = sum(n * n for n in ns)
    assert 1.5e7 < cells < 3.5e7


def test_study_instances_follow_section_3_1():
    """Static-drop study instances: La = 12000 with D = 0.4, rho = 300; the
    sharp-interface panel ties eps to the mesh by dx = sqrt(32) eps^(3/2)."""
    import math

    from paper_2205_05835_gb300 import studies as S

    plist, keys = S.study_instances("eps", (32, 64, 128), ("cdi", "sb"), ("eb", "csf", "lcsf"))
    assert len(plist) == 2 * 3 * 3 and keys[0] == ("cdi", "eb", 32)
    for p, (m, f, n) in zip(plist, keys):
        assert p["model"] == m and p["force"] == f and p["n"] == (n, n, 1)
        assert abs(p["sigma"] * p["rho_in"] * 2 * p["R"] / p["mu_in"] ** 2 - 12000) < 1e-9
        assert p["rho_in"] == p["rho_out"] == 300 and 2 * p["R"] == 0.4
        assert abs(math.sqrt(32) * p["eps"] ** 1.5 - 1.0 / n) < 1e-12
    assert abs(S.eps_of("eps", 32) - 1 / 32) < 1e-15 and S.eps_of("h", 256) == 1 / 32


def test_adjoint_workspace_and_validation(pf):
    """pf_adjoint_workspace_size: float64 CDI + EB only, size linear in the cells."""
    import pf_inputs as I

    p = pf.make_params(I.small_case(dim=2, n=32))
    b32 = pf.B.pf_adjoint_workspace_size(p)
    p64 = pf.make_params(I.small_case(dim=2, n=64))
    b64 = pf.B.pf_adjoint_workspace_size(p64)
    # 54 doubles per cell in 2D (plus 256-byte alignment of each array)
    assert 64 * 64 * 8 * 54 <= b64 <= 64 * 64 * 8 * 54 + 256 * 60
    assert b32 < b64
    for bad in (dict(precision="mixed"), dict(model="sb"), dict(force="csf")):
        q = pf.make_params(I.small_case(dim=2, n=32, **bad))
        with pytest.raises(pf.PFError) as e:
            pf.B.pf_adjoint_workspace_size(q)
        assert e.value.status == pf.B.PF_ERR_INVALID


def test_checkpoint_segments_cover_the_run(pf):
    from paper_2205_05835_gb300.adjoint import checkpoint_segments

    assert checkpoint_segments(500, 25) == [(s, 25) for s in range(0, 500, 25)]
    assert checkpoint_segments(10, 4) == [(0, 4), (4, 4), (8, 2)]
    assert checkpoint_segments(0, 3) == []
    for n, k in ((1, 1), (7, 3), (12, 5), (13, 13), (5, 9)):
        segs = checkpoint_segments(n, k)
        assert sum(c for _, c in segs) == n
        assert all(b == a + c for (a, c), (b, _) in zip(segs, segs[1:]))
    with pytest.raises(ValueError):
        checkpoint_segments(5, 0)


def test_momentum_transport_validation(pf):
    """Consistent transport needs the CDI model (its mass flux is the CDI flux)."""
    import pf_inputs as I

    ok = pf.make_params(I.small_case(dim=2, n=32, momentum="consistent"))
    assert pf.pf_workspace_size(ok) > 0
    for bad in (dict(momentum="consistent", model="sb"), dict(momentum="consistent", model="isodi"),
                dict(momentum="consistent", model="acdi")):
        q = pf.make_params(I.small_case(dim=2, n=32, **bad))
        with pytest.raises(pf.PFError) as e:
            pf.pf_workspace_size(q)
        assert e.value.status == pf.B.PF_ERR_INVALID
    q = pf.make_params(I.small_case(dim=2, n=32))
    q.momentum = 2
    with pytest.raises(pf.PFError):
        pf.pf_workspace_size(q)
    q = pf.make_params(I.small_case(dim=2, n=32, momentum="consistent"))
    with pytest.raises(pf.PFError):
        pf.B.pf_adjoint_workspace_size(q)


def test_wall_and_shape_validation(pf):
    """Free-slip walls in y: 2D with advective transport; the standing-wave
    shape needs them; the adjoint covers the periodic box only."""
    import pf_inputs as I

    ok = pf.make_params(I.standing_wave(n=32))
    assert ok.wall_y == 1 and ok.shape == 1
    assert pf.pf_workspace_size(ok) > 0
    bad = [I.standing_wave(n=32, momentum="consistent"),
           I.small_case(dim=3, n=16, wall_y=1),
           I.small_case(dim=2, n=32, shape="wave"),
           I.small_case(dim=2, n=32, wall_y=2)]
    for b in bad:
        with pytest.raises(pf.PFError) as e:
            pf.pf_workspace_size(pf.make_params(b))
        assert e.value.status == pf.B.PF_ERR_INVALID
    q = pf.make_params(I.small_case(dim=2, n=32))
    q.shape = 2
    with pytest.raises(pf.PFError):
        pf.pf_workspace_size(q)
    with pytest.raises(pf.PFError) as e:
        pf.B.pf_adjoint_workspace_size(ok)
    assert e.value.status == pf.B.PF_ERR_INVALID


def test_mg_coarse_cells_validation_and_autotune_keys(pf):
    """The coarse-solve threshold is 0 (default) or 16 .. 2^20; the autotuner's
    cache key separates what the best launch shape depends on."""
    import pf_inputs as I
    from paper_2205_05835_gb300 import autotune

    for v in (0, 16, 4096, 1 << 20):
        assert pf.pf_workspace_size(pf.make_params(I.small_case(dim=2, n=32,
                                                                mg_coarse_cells=v))) > 0
    for v in (8, (1 << 20) + 1, -1):
        with pytest.raises(pf.PFError) as e:
            pf.pf_workspace_size(pf.make_params(I.small_case(dim=2, n=32, mg_coarse_cells=v)))
        assert e.value.status == pf.B.PF_ERR_INVALID
    a = I.small_case(dim=2, n=64)
    assert autotune.signature(a) == autotune.signature(dict(a, sigma=3.0, R=0.2))
    for other in (dict(n=(80, 80, 1)), dict(precision="mixed"), dict(rho_out=0.01),
                  dict(use_graph=1), dict(force="csf"), dict(poisson_rtol=1e-8),
                  dict(inner_tol=1e-4)):
        assert autotune.signature(dict(a, **other)) != autotune.signature(a)
    # a shape tuned without the inner tolerance is not reused when it is asked for
    assert autotune.signature(a, tune_inner=True) != autotune.signature(a)
    assert {"mg_coarse_cells": 16384, "mg_pre": 1, "mg_post": 1} in autotune.CANDIDATES
    tuned = autotune.apply(a, {"choice": autotune.CANDIDATES[2]})
    assert tuned["mg_coarse_cells"] == 16384 and tuned["sigma"] == a["sigma"]


def test_autotune_keeps_defaults_within_the_margin(pf, monkeypatch):
    """Host logic of tune() with the timing replaced: a candidate must beat the
    library's defaults by more than MARGIN to be chosen, in the multigrid stage
    and in the 3D mixed tile stage; a clearly faster one is chosen."""
    from paper_2205_05835_gb300 import autotune

    def run(times, p):
        def fake(pf_, p_, cand, steps, warm):
            key = tuple(sorted(cand.items()))
            return times.get(key, 1.0)
        monkeypatch.setattr(autotune, "_time_candidate", fake)
        autotune._cache.clear()
        return autotune.tune(p, candidates=cands)["choice"]

    d = autotune.DEFAULT_SHAPE
    other = {"mg_coarse_cells": 1024, "mg_pre": 2, "mg_post": 2}
    cands = (d, other)
    k = lambda c: tuple(sorted(c.items()))  # noqa: E731
    p2 = {"dim": 2, "n": (64, 64, 1), "precision": "mixed", "rho_in": 10.0, "rho_out": 1.0}
    # 0.5 % faster: keep the defaults; 3 % faster: take the candidate
    assert run({k(d): 1.0, k(other): 0.995}, p2) == d
    assert run({k(d): 1.0, k(other): 0.97}, p2) == other
    # 3D mixed: tile shapes are tried after the shape, with the same margin
    p3 = dict(p2, dim=3, n=(64, 64, 64))
    t2 = dict(d, sweep_tile=2)
    t3 = dict(d, sweep_tile=3)
    assert run({k(d): 1.0, k(other): 1.2, k(t2): 0.995, k(t3): 1.1}, p3) == d
    assert run({k(d): 1.0, k(other): 1.2, k(t2): 0.98, k(t3): 0.95}, p3) == t3
