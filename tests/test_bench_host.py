"""Host-side pieces of bench.py that need no GPU: the roofline arithmetic over the
library's per-class counters and the material-estimation workloads' sizes."""
import numpy as np
import pytest

import bench
from paper_2301_01396_gb300 import scenes


def test_class_roofline_picks_the_dominant_class():
    stats = {
        "fwd_phase": {"launches": 8, "units": 800, "ms": 4.0, "timed_launches": 8, "alg_bytes": 8.0e9},
        "vjp_phase": {"launches": 8, "units": 800, "ms": 6.0, "timed_launches": 8, "alg_bytes": 12.0e9},
        "predict": {"launches": 2, "units": 20, "ms": 0.1, "timed_launches": 2, "alg_bytes": 1.0e6},
        "other": {"launches": 1, "units": 1, "ms": 0.0, "timed_launches": 0, "alg_bytes": 0.0},
    }
    roof, cls, brk = bench.class_roofline(stats, steps=2)
    assert roof["kernel"] == "vjp_phase"
    # 1.5e9 B per launch over 0.75 ms per launch = 2000 GB/s
    assert roof["achieved"] == pytest.approx(2000.0)
    assert roof["bytes_per_unit"] == pytest.approx(1.5e7)
    assert roof["frac"] == pytest.approx(2000.0 / roof["peak"], rel=1e-3)
    assert cls["fwd_phase"]["gbs"] == pytest.approx(2000.0)
    assert brk["vjp_phase"] == pytest.approx(3.0) and "other" not in brk


@pytest.mark.parametrize("kind, V, rows", [("tets", 35937, 327680), ("tets-coupled", 35937, 327680),
                                           ("membrane", 65536, 129540 + 3 * 130050)])
def test_material_workload_sizes(kind, V, rows):
    sc = bench.material_scene(kind)
    assert sc.V == V and sc.m + 3 * sc.n_memb == rows
    scenes.validate_coloring(sc)
    if kind == "tets-coupled":
        assert sc.tet_coupled and sc.n_colors == 40
    if kind == "membrane":
        assert sc.collider_flags == scenes.COLLIDE_PLANE and sc.plane_h == -0.6
        assert np.all(sc.inv_mass > 0)


def test_reference_arm_line_keeps_the_contract():
    """The reference arm (the oracle on the host cores) prints one line with the keys the
    driver reads; its e2e moves no bytes and its cpu_baseline describes the same run."""
    class Args:
        cpu_window, warmup, steps = 8, 0, 1

    d = bench.run_reference(Args, 1, 0)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert bench.run_reference(Args, 2, 1) is None
