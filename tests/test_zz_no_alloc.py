"""alm_eval_static: the actuator-line evaluation for callers that cannot
allocate device memory (a real-time turbine-controller loop, or code inside
another framework that owns the memory pool, where cudaMalloc/cudaFree may
synchronise the device or are not allowed).  It keeps its scratch in a
static device block.

Checked through the C ABI against the lattice's own evaluation
(alm_get_loads) on two calls in a row with different flow states, at an even
and an odd step, with the device's free memory unchanged by the second call.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2402_13171_gb300 import inputs as I
from paper_2402_13171_gb300 import lbm

pytestmark = pytest.mark.gpu

C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)])
W1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
W = np.array([W1[c[0]] * W1[c[1]] * W1[c[2]] for c in C])


def _desc(t):
    d = lbm.AlmTurbineDesc()
    keep = {k: np.ascontiguousarray(t[k], dtype=np.float64) for k in ("alpha", "cl", "cd")}
    for a in range(3):
        d.hub[a] = t["hub"][a]
    d.radius = t["radius"]
    d.n_blades = t["n_blades"]
    d.n_elements = t["n_elements"]
    d.epsilon = t["epsilon"]
    d.omega = t["omega"]
    d.yaw, d.pitch, d.theta0 = t["yaw"], t["pitch"], t["theta0"]
    d.chord_root, d.chord_tip = t["chord_root"], t["chord_tip"]
    d.twist = None
    d.n_polar = keep["alpha"].size
    d.alpha = keep["alpha"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.cl = keep["cl"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.cd = keep["cd"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.regularisation = lbm.REGULARISATION[t["kernel"]]
    d.tip_loss = int(t["tip_loss"])
    return d, keep


def _static_fn():
    L = lbm.load()
    fn = L.alm_eval_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(lbm.AlmTurbineDesc), ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn


@pytest.mark.parametrize("kernel,tip_loss", [("gauss", False), ("roma", True)])
def test_static_alm_matches_lattice_on_two_calls(kernel, tip_loss):
    """Two calls in a row, at an even and an odd step (the two halves of the
    block's double buffers), on two different flow states: each equals the
    lattice's own evaluation at that step, and from the second call on the
    device's free memory does not change (the call allocates nothing)."""
    import torch
    from paper_2402_13171_gb300 import build
    build.build()
    fn = _static_fn()
    nx, ny, nz = 64, 40, 40
    dom, turb = I.single_turbine_case(nx, ny, nz, diameter=16.0, elements_per_blade=8, seed=31, kernel=kernel,
                                      tip_loss=tip_loss)
    body = (2e-6, 0.0, -1e-6)
    g = lbm.Lattice.create(nx, ny, nz, nu=dom["nu"], bc=("periodic",) * 3, body_force=body)
    g.add_turbine(**turb)
    desc, keep = _desc(turb)
    n_el = turb["n_blades"] * turb["n_elements"]
    bodyc = (ctypes.c_double * 3)(*body)
    stream = torch.cuda.Stream()
    ef = torch.empty(3 * n_el, dtype=torch.float32, device="cuda")
    ep = torch.empty(3 * n_el, dtype=torch.float32, device="cuda")
    ld = torch.empty(2, dtype=torch.float64, device="cuda")
    for call, (seed, step) in enumerate(((1, 0), (2, 1))):
        rho, u, fneq = I.random_state(nx, ny, nz, seed=seed, u_mean=(0.05, 0.0, 0.0), du=0.01, drho=0.005)
        g.set_step(0)
        g.init_fields(rho, u, fneq)
        g.set_step(step)           # the lattice's actuator line of `step`, from this state
        # the caller's own copy of the lattice's FP32 offsets f - w
        h = torch.tensor((g.pdfs() - W[:, None, None, None]).astype(np.float32), device="cuda").contiguous()
        if step > 0:
            g.step(1)              # the loads of step `step` are read after it ran
        th, tq, ef_ref, ep_ref = g.loads(0, elements=True)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        s = fn(h.data_ptr(), nx, ny, nz, bodyc, ctypes.byref(desc), step, ef.data_ptr(), ep.data_ptr(),
               ld.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert s == 0, lbm.STATUS.get(s, s)
        stream.synchronize()
        if call > 0:
            assert torch.cuda.mem_get_info()[0] == free0
        np.testing.assert_allclose(ep.cpu().numpy().reshape(-1, 3), ep_ref, atol=2e-5)
        np.testing.assert_allclose(ef.cpu().numpy().reshape(-1, 3), ef_ref, rtol=0,
                                   atol=1e-7 + 5e-5 * np.abs(ef_ref).max())
        loads = ld.cpu().numpy()
        assert loads[0] == pytest.approx(th, rel=5e-5)
        assert loads[1] == pytest.approx(tq, rel=5e-5)
    # beyond the static limit: rejected before anything runs
    big = dict(turb, n_elements=400)
    bdesc, bkeep = _desc(big)
    assert fn(h.data_ptr(), nx, ny, nz, bodyc, ctypes.byref(bdesc), 0, ef.data_ptr(), ep.data_ptr(), ld.data_ptr(),
              ctypes.c_void_p(stream.cuda_stream)) == 1
    g.destroy()
