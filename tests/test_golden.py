"""Values the paper prints, held as fixtures under tests/golden/.

* Sec. 4 performance model: the bytes per cell update, the bandwidth ceiling
  P_max = b_S / n_b, the A100 lightspeed and the measured fractions are
  recomputed with the functions bench.py uses for its roofline.
* Sec. 5 operating points: the oracle's blade kinematics, driven with
  Omega = TSR U / R, move the blade tips at TSR times the wind speed, and the
  three cases correspond to one rotor speed within the rounding of the printed
  tip-speed ratios.
"""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
sys.path.insert(0, ROOT)


def _read(name):
    scalars, rows = {}, []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        if len(parts) == 2 and not _isnum(parts[0]):
            scalars[parts[0]] = float(parts[1])
        else:
            rows.append(parts)
    return scalars, rows


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


def test_performance_model_of_sec4():
    import bench
    sc, rows = _read("performance_model_sec4.txt")
    assert bench.bytes_per_cell_update(force_components=3) == sc["n_b_bytes"]
    # the fused in-kernel gather reads no force field
    assert bench.bytes_per_cell_update() == 216
    assert bench.bytes_per_cell_update(elem_bytes=2) == 108
    l = bench.lightspeed(1713.0, sc["n_f_flops"], sc["a100_peak_tflops"] * 1e3, sc["n_b_bytes"])
    assert round(l, 4) == sc["a100_lightspeed"]
    for name, bs, pmax, _without, with_t, ratio in rows:
        bs, pmax, with_t, ratio = float(bs), float(pmax), float(with_t), float(ratio)
        assert bench.max_mlups(bs, sc["n_b_bytes"]) == pytest.approx(pmax, abs=0.05), name
        assert 100 * with_t / bench.max_mlups(bs, sc["n_b_bytes"]) == pytest.approx(ratio, abs=0.05), name


def test_operating_points_of_sec5_tip_speed():
    import oracle as O
    sc, rows = _read("newmexico_operating_points.txt")
    R = sc["diameter_m"] / 2
    omegas = []
    for U, tsr in ((float(a), float(b)) for a, b in rows):
        omega = tsr * U / R
        omegas.append(omega)
        # the oracle's blade kinematics (Algorithm 2), lengths in metres: every
        # element of every blade moves at omega r, so the tip (r = R) moves at
        # omega R = TSR U
        spec = O.TurbineSpec(hub=(40.0, 40.0, 40.0), radius=R, n_blades=3, n_elements=4, epsilon=2.0,
                             omega=omega, alpha=np.radians(np.linspace(-180, 180, 3601)), cl=np.zeros(3601),
                             cd=np.zeros(3601), theta0=0.3)
        for b in range(3):
            for k in range(4):
                kin = O.element_kinematics(spec, 7, b, k)
                r = np.linalg.norm(kin["pos"] - np.array([40.0, 40.0, 40.0]))
                assert r == pytest.approx((k + 0.5) * R / 4, rel=1e-12)
                assert np.linalg.norm(kin["vel"]) == pytest.approx(omega * r, rel=1e-12)
        assert omega * R / U == pytest.approx(tsr, rel=1e-12)
    # one rotor speed (the printed ratios are rounded): spread below 5 %
    assert (max(omegas) - min(omegas)) / np.mean(omegas) < 0.05
