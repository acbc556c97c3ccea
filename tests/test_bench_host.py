"""Host-side pieces of bench.py: the whole-step roofline arithmetic and the
multi-core oracle baseline of the batch workload (CPU only)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_step_roofline_sums_finest_classes(bench):
    # two classes on a 1000-cell 3D float32 grid: 16 B/cell x 10 launches and
    # 20 B/cell x 5 (the direction product reads the cell densities, not the
    # three face arrays: 28 B/cell in float32 with face arrays, 2D)
    prof = {"mg_gs_level0": (10, 2.0), "cg_dir_spmv": (5, 1.0), "mg_restrict": (50, 3.0)}
    r = bench.step_roofline(prof, 1000, 3, 4, ms_total=4.0, ms_host=8.0, peak=100.0)
    want_bytes = 16 * 1000 * 10 + 20 * 1000 * 5
    assert bench.algo_bytes_per_cell("cg_dir_spmv", 2, 4) == 24
    assert bench.algo_bytes_per_cell("cg_dir_spmv", 3, 8) == 56
    assert r["bytes"] == want_bytes
    assert r["achieved"] == pytest.approx(want_bytes / 4e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 100.0)
    assert r["their_time_share"] == pytest.approx(3.0 / 8.0)   # the coarse class is left out
    assert "mg_restrict" not in r["classes"]
    assert bench.step_roofline({}, 1000, 3, 4, 4.0, 8.0, 100.0) is None


def test_cpu_batch_rate_runs_the_oracle_on_a_pool(bench):
    import pf_inputs as I

    plist = I.batch_manifest()
    small = [p for p in plist if p["n"][0] <= 64][:2]
    assert len(small) == 2
    v, cores, desc = bench.cpu_batch_rate(small, steps=1, max_n=64)
    assert v > 0 and 1 <= cores <= 2 and "spawned" in desc


def test_multilevel_classes_in_the_step_roofline(bench):
    """The multigrid levels follow the library's halving rule, and the classes
    that span several levels add their bytes per V-cycle times the V-cycles."""
    assert bench.mg_levels((384, 384, 384), 3) == [384 ** 3, 192 ** 3, 96 ** 3, 48 ** 3, 24 ** 3]
    assert bench.mg_levels((256, 256, 1), 2) == [256 ** 2, 128 ** 2]
    lv = bench.mg_levels((64, 64, 64), 3)
    cb = bench.coarse_class_bytes(lv, 3, 4)
    # restriction: x, f, rho (12 B) + 1/8 coarse write on the finest level and
    # level 1 (densities), x, f and three face arrays below
    assert cb["mg_restrict"] == lv[0] * 12.5 + lv[1] * 12.5
    # sweeps of level 1 from its densities: 12 B from zero, 16 B from x_in
    assert cb["mg_gs_coarse_levels"] == lv[1] * (12 + 16)
    lv4 = bench.mg_levels((384, 384, 384), 3)
    cb4 = bench.coarse_class_bytes(lv4, 3, 4)
    assert cb4["mg_restrict"] == sum(c * (12.5 if i <= 1 else 20.5) for i, c in enumerate(lv4))
    assert cb["mg_prolong"] == sum(c * 8.5 for c in lv)
    prof = {"mg_gs_level0": (10, 2.0), "mg_restrict": (20, 1.0), "mg_prolong": (20, 1.0),
            "mg_gs_coarse_levels": (20, 1.0), "mg_coarse_vcycle": (10, 0.5)}
    r0 = bench.step_roofline(prof, lv[0], 3, 4, 4.0, 8.0, 100.0)
    r1 = bench.step_roofline(prof, lv[0], 3, 4, 4.0, 8.0, 100.0, levels=lv, vcycles=10)
    assert r1["bytes"] == r0["bytes"] + 10 * sum(cb.values())
    assert "mg_prolong" in r1["classes"] and "mg_coarse_vcycle" not in r1["classes"]
