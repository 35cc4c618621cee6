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


def test_non_finite_state_sets_numeric_error_and_stays_sticky():
    """The FP64 diagnostic sums double as a NaN/Inf watchdog: a NaN placed in
    one population of the initial state (a host input, no GPU fault) spreads
    through the collision, the next diagnostic sum is non-finite, and the next
    synchronising call reports LBM_ERR_NUMERIC -- as does every later call."""
    dom = dict(nx=24, ny=12, nz=10, nu=0.02)
    rho, u, fneq = I.random_state(24, 12, 10, seed=17)
    fneq[5, 3, 4, 7] = np.nan
    g = gpu_lattice(dom, diag_every=1)
    g.init_fields(rho, u, fneq)
    g.step(2)
    with pytest.raises(lbm.LbmError, match="non-finite state"):
        g.sync()
    for call in (lambda: g.step(1), g.moments, g.diagnostics):
        with pytest.raises(lbm.LbmError, match="non-finite state"):
            call()
    g.destroy()
    # the same input without the NaN runs clean
    fneq[5, 3, 4, 7] = 0.0
    h = gpu_lattice(dom, diag_every=1)
    h.init_fields(rho, u, fneq)
    h.step(2)
    h.sync()
    assert np.all(np.isfinite(h.diagnostics()[0]))
    h.destroy()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_staged_copy_wait_timeout_is_reported(storage):
    """The staged step's waits on its own TMA row copies are bounded.  With the
    bound set to 0 cycles every wait gives up before it looks (the copies
    themselves are valid and complete a little later); the kernel sets
    the timeout bit, waits with the default bound for the copies it still has
    in flight, and returns.  The next synchronising call reports
    LBM_ERR_TIMEOUT, sticky; a fresh lattice in the same process runs clean."""
    dom, turb = I.single_turbine_case(128, 48, 40, diameter=16.0, elements_per_blade=8, seed=5)
    g = gpu_lattice(dom, storage=storage, tile=(64, 1, 1, 1))
    g.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
    g.add_turbine(**turb)
    assert g.tile()[3] == 1
    g.step(2)
    g.sync()                          # the default bound: no timeout
    g.set_wait_limit(0)
    g.step(2)
    with pytest.raises(lbm.LbmError, match="device wait timed out"):
        g.sync()
    with pytest.raises(lbm.LbmError, match="device wait timed out"):
        g.step(1)
    g.destroy()
    bad = gpu_lattice(dom, storage=storage, tile=(64, 1, 1, 1))
    with pytest.raises(lbm.LbmError, match="invalid argument"):
        bad.set_wait_limit(-1)
    bad.destroy()
    h = _case()
    h.step(4)
    h.sync()
    h.destroy()
