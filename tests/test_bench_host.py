"""Host logic of the benchmark that decides what a run reports: the clock
record that accepts or rejects a run, the algorithmic byte counts behind
each class's roofline, and the class roofline arithmetic."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_lines_give_median_max_and_the_reasons_seen():
    lines = [
        "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
        "1995, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1100.0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = bench.parse_clock_lines(lines)
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.parse_clock_lines(["1500, 2070, 1400, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clock_lines([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


@pytest.mark.parametrize("dims,model", [(2, "komegasst"), (2, "kepsilon"), (3, "kepsilon"), (2, "laminar")])
def test_byte_model_invariants(dims, model):
    mixed = bench.class_bytes_per_sweep(dims, True, model, 5)
    fp64 = bench.class_bytes_per_sweep(dims, False, model, 5)
    assert set(mixed) == set(fp64)
    # the solves' own words are FP32 on the mixed path (its assembly adds
    # FP32 defects, so only the inner sweeps and the pressure solve shrink)
    for k in ("mom_smooth", "pcg") + (("scal_smooth",) if model != "laminar" else ()):
        assert 0 < mixed[k] < fp64[k], k
    # the pressure class grows by the same amount per CG iteration
    b = [bench.class_bytes_per_sweep(dims, True, model, n)["pcg"] for n in (3, 4, 5)]
    assert b[2] - b[1] == pytest.approx(b[1] - b[0]) and b[1] > b[0]
    # one gradient launch per sweep: flags, the velocity, its D x D gradient
    assert fp64["grad_u"] == 2 + dims * 8 + dims * dims * 8
    # more inner sweeps cost more
    assert bench.class_bytes_per_sweep(dims, True, model, 5, n_u=3)["mom_smooth"] > mixed["mom_smooth"]
    if model != "laminar":
        assert {"turb_prep", "scal_asm", "scal_smooth", "turb_final"} <= set(fp64)
    else:
        assert "turb_prep" not in fp64


def test_three_dimensions_move_more_bytes_per_cell():
    b2 = bench.class_bytes_per_sweep(2, True, "kepsilon", 5)
    b3 = bench.class_bytes_per_sweep(3, True, "kepsilon", 5)
    for k in b2:
        assert b3[k] >= b2[k], k
    for k in ("grad_u", "mom_asm", "mom_smooth", "hbya", "update", "scal_asm", "scal_smooth"):
        assert b3[k] > b2[k], k


def test_class_roofline_arithmetic():
    prof = {"pcg": (3690.0, 10), "update": (319.0, 10), "idle": (0.0, 0)}
    out = bench.class_roofline(prof, 10, 262144, {"pcg": 808.9, "update": 122.0}, 6801.7)
    assert "idle" not in out
    assert out["pcg"]["us_per_sweep"] == 369.0
    gbs = 808.9 * 262144 / 369.0e-6 / 1e9
    assert out["pcg"]["gbs"] == pytest.approx(gbs, abs=0.05)
    assert out["pcg"]["frac"] == pytest.approx(gbs / 6801.7, abs=1e-4)
    assert out["pcg"]["share"] + out["update"]["share"] == pytest.approx(1.0, abs=1e-3)
