"""The seeded input recipe of the workloads (what the benchmark and the tests
feed both the CUDA path and the oracle): reproducible, within the stated
ranges, and valid for the solver's host checks."""
import math

import numpy as np
import pytest

from paper_2402_13171_gb300 import inputs as I


def test_single_rotor_workload_recipe():
    dom, t = I.single_turbine_case()
    assert (dom["nx"], dom["ny"], dom["nz"]) == (256, 128, 128)
    assert dom["bc"] == ("inout", "periodic", "periodic") and dom["noise_rel"] == 0.01
    assert t["hub"] == (64.0, 64.0, 64.0) and t["radius"] == 16.0
    assert t["n_blades"] == 3 and t["n_elements"] == 40 and t["epsilon"] == 2.0
    assert t["omega"] == pytest.approx(0.01875, rel=1e-15)          # TSR 6 at U = 0.05: TSR U / R
    assert (t["chord_root"], t["chord_tip"]) == (2.0, 1.0)
    assert t["kernel"] == "gauss" and t["tip_loss"] is False


def test_synthetic_polars():
    a, cl, cd = I.synthetic_polars()
    assert a.size == 3601 and a[0] == -math.pi and a[-1] == math.pi
    np.testing.assert_allclose(np.diff(a), math.radians(0.1), rtol=1e-9)
    small = np.abs(2 * math.pi * a) < 1.2
    np.testing.assert_array_equal(cl[small], 2 * math.pi * a[small])
    assert np.all(np.abs(cl) <= 1.2) and cl[0] == -1.2 and cl[-1] == 1.2
    np.testing.assert_allclose(cd, 0.01 + 0.02 * a ** 2, rtol=0, atol=0)


def test_batch_sweep_recipe_and_rotor_support():
    """The 16 lattices of the batched sweep: sizes multiples of 8 in the stated
    ranges (71,866,368 cells in all), TSR in [3, 9], inflow in [0.03, 0.06], and
    every rotor's force support, hub +- (R + 3 eps + 1), inside [1, n-2]."""
    cases = I.batch_instances(16)
    again = I.batch_instances(16)
    total = 0
    for (d, t), (d2, t2) in zip(cases, again):
        assert d == d2 and t["hub"] == t2["hub"] and t["omega"] == t2["omega"]
        nx, ny, nz = d["nx"], d["ny"], d["nz"]
        total += nx * ny * nz
        assert nx % 8 == ny % 8 == nz % 8 == 0
        assert 128 <= nx <= 384 and 96 <= ny <= 160 and 96 <= nz <= 160
        R, U = t["radius"], d["u_ref"][0]
        assert 8.0 <= R <= 20.0 and 2 * R <= 0.5 * min(ny, nz) - 16 + 1e-12
        assert 3.0 <= t["omega"] * R / U <= 9.0 and 0.03 <= U <= 0.06
        assert t["hub"] == (nx / 4.0, ny / 2.0, nz / 2.0)
        ext = R + 3 * t["epsilon"] + 1
        for a, n in enumerate((nx, ny, nz)):
            reach = ext if a else 3 * t["epsilon"] + 1      # the rotor faces x (yaw 0)
            assert math.floor(t["hub"][a] - reach) >= 1 and math.ceil(t["hub"][a] + reach) <= n - 2
    assert total == 71866368


def test_random_state_is_seeded_and_bounded():
    r1, u1, f1 = I.random_state(9, 7, 5, seed=3, u_mean=(0.05, 0, 0), du=0.01, drho=0.002, fneq_amp=2e-4)
    r2, u2, f2 = I.random_state(9, 7, 5, seed=3, u_mean=(0.05, 0, 0), du=0.01, drho=0.002, fneq_amp=2e-4)
    np.testing.assert_array_equal(r1, r2)
    np.testing.assert_array_equal(f1, f2)
    assert r1.shape == (5, 7, 9) and u1.shape == (3, 5, 7, 9) and f1.shape == (27, 5, 7, 9)
    assert f1.dtype == np.float32
    assert np.all(np.abs(r1 - 1) <= 0.002) and np.all(np.abs(u1[0] - 0.05) <= 0.01)
    assert np.all(np.abs(f1[13]) <= 2e-4 * 0.3 * (1 + 1e-6)) and np.all(np.abs(f1[0]) <= 2e-4 * 0.005 * (1 + 1e-6))
    r3, _, _ = I.random_state(9, 7, 5, seed=4)
    assert not np.array_equal(r1, r3)


def test_unequal_polar_table_and_twist():
    a, cl, cd = I.nonuniform_polars()
    assert a[0] == pytest.approx(-math.pi) and a[-1] == pytest.approx(math.pi) and np.all(np.diff(a) > 0)
    d = np.degrees(np.diff(a))
    assert d.min() < 0.3 and d.max() == pytest.approx(5.0)
    np.testing.assert_allclose(cl, np.clip(2 * math.pi * a, -1.2, 1.2), rtol=0, atol=0)
    tw = I.blade_twist(8)
    assert tw.shape == (8,) and np.all(np.diff(tw) < 0) and 0.02 < tw[-1] < tw[0] < 0.2


def test_small_farm_recipe_and_rotor_supports():
    """The scaled-down farm: log-law inflow referenced to hub height, free-slip
    bottom and top, periodic y, two yawed rotors whose force supports
    (hub +- (R sqrt(1 - e_axis_a^2) + 3 eps + 1)) lie inside [1, n - 2]."""
    dom, turbs = I.small_farm_case()
    assert dom["bc"] == ("inout", "periodic", "freeslip") and dom["inflow_kind"] == 1
    assert dom["z_ref"] == dom["nz"] / 2 and len(turbs) == 2
    n = (dom["nx"], dom["ny"], dom["nz"])
    for t in turbs:
        assert 0 < t["yaw"] < math.radians(10) and t["hub"][2] == dom["z_ref"]
        ea = (math.cos(t["yaw"]), math.sin(t["yaw"]), 0.0)
        for a in range(3):
            ext = t["radius"] * math.sqrt(max(0.0, 1 - ea[a] ** 2)) + 3 * t["epsilon"] + 1
            assert math.floor(t["hub"][a] - ext) >= 1 and math.ceil(t["hub"][a] + ext) <= n[a] - 2
    prof = I.log_law_profile(dom["nz"], 0.05, 0.1, dom["z_ref"])
    assert prof[int(dom["z_ref"] - 0.5)] < 0.05 < prof[int(dom["z_ref"] + 0.5)]
