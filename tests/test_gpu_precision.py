"""16-bit PDF storage against the FP64 oracle on a 128^3 crop of the rotor case.

A 128^3 lattice with velocity inlet / zero-gradient outlet holds the rotor of
the 256x128x128 workload (D = 32 at (32, 64, 64), 3 x 40 elements, eps = 2);
the same seeded run is made with PDFs stored as FP32, BF16 and FP16 offsets and
by the oracle.  Bounds: FP32 at the laminar parity tolerance; BF16 (8-bit
mantissa) and FP16 (11-bit) at their per-step rounding of ~0.05-sized
offsets times the horizon.
"""
import numpy as np
import pytest

from paper_2402_13171_gb300 import inputs as I
from cases import setup_pair

pytestmark = pytest.mark.gpu


def test_storage_precision_on_128_crop():
    dom, turb = I.single_turbine_case(128, 128, 128, hub=(32.0, 64.0, 64.0))
    steps = 40
    g32, s = setup_pair(dom, [turb], inflow=True)
    s.step(steps)
    _, uo = s.moments()
    errs = {}
    for storage in ("fp32", "bf16", "fp16"):
        g = g32 if storage == "fp32" else setup_pair(dom, [turb], inflow=True, storage=storage)[0]
        g.step(steps)
        _, ug = g.moments()
        d = ug - uo
        errs[storage] = (float(np.abs(d).max()), float(np.sqrt(np.mean(d ** 2))))
        print(f"{storage}: max|du| {errs[storage][0]:.3e}  rms {errs[storage][1]:.3e}  (U = 0.05, {steps} steps)")
        g.destroy()
    assert errs["fp32"][0] <= 1e-6
    assert errs["fp16"][0] < 2e-4
    assert errs["bf16"][0] < 2e-3
    assert errs["fp16"][1] < errs["bf16"][1]
