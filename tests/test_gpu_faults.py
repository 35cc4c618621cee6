"""Failure paths exercised by host-side fault injection (LBM_FAULT), with no
fault on the GPU: a failed device allocation, a failed graph capture and a
failed step.  Each error is reported through the status of the call, stays
sticky on the context, and leaves the steps before it intact."""
import numpy as np
import pytest

from paper_2402_13171_gb300 import inputs as I
from paper_2402_13171_gb300 import lbm
from cases import gpu_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_13171_gb300 import build
    build.build()


def _case():
    dom, turb = I.single_turbine_case(64, 40, 40, diameter=16.0, elements_per_blade=8, seed=5)
    g = gpu_lattice(dom)
    g.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
    g.add_turbine(**turb)
    return g


def test_injected_allocation_failure(monkeypatch):
    monkeypatch.setenv("LBM_FAULT", "alloc")
    with pytest.raises(lbm.LbmError, match="out of device memory"):
        lbm.Lattice.create(32, 16, 16)
    monkeypatch.delenv("LBM_FAULT")
    g = lbm.Lattice.create(32, 16, 16)   # the process is unharmed
    g.step(3)
    g.sync()
    g.destroy()


def test_injected_step_failure_is_sticky(monkeypatch):
    ref, g = _case(), _case()
    ref.step(5)
    monkeypatch.setenv("LBM_FAULT", "step:5")
    g.step(5)                             # steps 0..4 run
    np.testing.assert_array_equal(g.pdfs(), ref.pdfs())
    with pytest.raises(lbm.LbmError, match="step 5 failed"):
        g.step(3)
    monkeypatch.delenv("LBM_FAULT")
    with pytest.raises(lbm.LbmError, match="CUDA error"):
        g.moments()                       # sticky until destroy
    g.destroy()
    ref.destroy()


def test_injected_capture_failure(monkeypatch):
    g = _case()
    monkeypatch.setenv("LBM_FAULT", "capture")
    g.step(1)                             # a single step needs no graph
    with pytest.raises(lbm.LbmError, match="graph capture failed"):
        g.step(8)
    g.destroy()
