"""Host-side argument checks of the C ABI, which run before any CUDA call:
lattice sizes (including the 32-bit plane-offset limit 27 N < 2^31), boundary
codes, viscosity, tiles, batches whose members disagree, the in-place scheme's
limits, and the rotor of the allocation-free actuator-line entry point."""
import ctypes

import pytest

from paper_2402_13171_gb300 import lbm

INVALID_ARG, UNSUPPORTED = 1, 7


def _create(**kw):
    L = lbm.load()
    nx, ny, nz = kw.pop("nx", 16), kw.pop("ny", 16), kw.pop("nz", 16)
    cfg = lbm.make_config(nx, ny, nz, **kw)
    h = ctypes.c_void_p()
    return L.lbm_create(ctypes.byref(cfg), ctypes.byref(h))


@pytest.mark.parametrize("kw", [
    dict(nx=0), dict(ny=-3), dict(nz=65536),
    # 27 N must stay below 2^31: 79,536,431 cells at most
    dict(nx=1024, ny=384, nz=203),
    dict(collision=5), dict(storage=3), dict(nu=0.0), dict(nu=-0.1), dict(nu=float("nan")),
    dict(bc=("periodic", "inout", "periodic")), dict(bc=("periodic", "periodic", "inout")),
    dict(bc=(7, 0, 0)), dict(nx=1, bc=("inout", "periodic", "periodic")),
    dict(diag_every=-1),
    dict(tile=(16, 4)), dict(tile=(48, 2)), dict(tile=(64, 8)), dict(tile=(32, 2, 65)), dict(tile=(32, -1)),
    dict(tile=(32, 4, 1, 3)), dict(tile=(32, 4, 1, -1)),
])
def test_invalid_configurations_are_rejected_on_the_host(kw):
    assert _create(**kw) == INVALID_ARG


def test_size_limit_is_exact():
    # 27 * 1024 * 384 * 202 = 2,144,600,064 < 2^31 passes the size check (and
    # then needs a device); one more plane does not
    assert 27 * 1024 * 384 * 202 < 2 ** 31 <= 27 * 1024 * 384 * 203
    assert _create(nx=1024, ny=384, nz=203) == INVALID_ARG


def test_batch_members_must_agree():
    L = lbm.load()
    arr = (lbm.LbmConfig * 2)()
    arr[0] = lbm.make_config(16, 16, 16, storage="fp32")
    arr[1] = lbm.make_config(24, 16, 16, storage="bf16")
    hs = (ctypes.c_void_p * 2)()
    assert L.lbm_batch_create(2, arr, hs) == UNSUPPORTED
    arr[1] = lbm.make_config(24, 16, 16, nu=-1.0)
    assert L.lbm_batch_create(2, arr, hs) == INVALID_ARG
    assert L.lbm_batch_create(0, arr, hs) == INVALID_ARG


def test_status_strings_cover_every_code():
    L = lbm.load()
    for code in range(8):
        assert L.lbm_status_string(code)


def _static_desc(**over):
    import numpy as np
    from paper_2402_13171_gb300 import inputs as I
    t = I.single_turbine(64, 40, 40, diameter=16.0, elements_per_blade=8)
    keep = [np.ascontiguousarray(t[k], dtype=np.float64) for k in ("alpha", "cl", "cd")]
    d = lbm.AlmTurbineDesc()
    for a in range(3):
        d.hub[a] = t["hub"][a]
    d.radius, d.n_blades, d.n_elements = t["radius"], t["n_blades"], t["n_elements"]
    d.epsilon, d.omega = t["epsilon"], t["omega"]
    d.chord_root, d.chord_tip = t["chord_root"], t["chord_tip"]
    d.n_polar = keep[0].size
    d.alpha, d.cl, d.cd = (k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k in keep)
    for k, v in over.items():
        setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("over", [dict(regularisation=2), dict(regularisation=-1),
                                  dict(tip_loss=2), dict(tip_loss=-1),
                                  dict(epsilon=0.0), dict(epsilon=6.0), dict(radius=0.0),
                                  dict(hub=(16.0, 10.9, 20.0), regularisation=1),
                                  # 3 x 1431655766 wraps to 2 in 32-bit arithmetic
                                  dict(n_blades=3, n_elements=1431655766), dict(n_blades=1025, n_elements=1),
                                  dict(hub=(float("nan"), 20.0, 20.0)), dict(yaw=float("nan")),
                                  dict(omega=float("inf")), dict(theta0=float("nan")), dict(pitch=float("-inf")),
                                  dict(chord_tip=float("nan"))])
def test_static_alm_rejects_bad_rotors_on_the_host(over):
    """alm_eval_static checks its rotor before any CUDA call: an unknown
    regularisation or tip-loss code, a Gaussian width outside [0.5, 5], a zero radius,
    a Roma support (hub +- (R + 3/2 + 1)) that leaves [1, n-2], blade and element
    counts whose product exceeds the static limit (also where the 32-bit product
    would wrap), and non-finite inputs (a NaN hub passes the support test, whose
    comparisons are all false for NaN)."""
    L = lbm.load()
    fn = L.alm_eval_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(lbm.AlmTurbineDesc), ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    hub = over.pop("hub", None)
    d, keep = _static_desc(**over)
    if hub is not None:
        for a in range(3):
            d.hub[a] = hub[a]
    # the PDF, force and load pointers are only tested for NULL before the checks fail
    dummy = ctypes.c_void_p(256)
    assert fn(dummy, 64, 40, 40, None, ctypes.byref(d), 0, dummy, None, dummy, None) == INVALID_ARG


@pytest.mark.parametrize("kw,code", [
    (dict(inplace=True, tile=(32, 4, 2)), UNSUPPORTED),
    (dict(inplace=True, tile=(64, 1, 1, 1)), UNSUPPORTED),
])
def test_inplace_scheme_limits_are_checked_on_the_host(kw, code):
    """The in-place (AA) scheme takes single-plane direct tiles only;
    marching or staged tiles are refused at creation."""
    assert _create(**kw) == code


def test_inplace_flag_must_be_boolean():
    L = lbm.load()
    cfg = lbm.make_config(16, 16, 16)
    cfg.inplace = 2
    h = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(cfg), ctypes.byref(h)) == INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("over", [dict(n_blades=3, n_elements=1431655766), dict(hub=(float("nan"), 20.0, 20.0)),
                                  dict(yaw=float("nan")), dict(omega=float("nan"))])
def test_add_turbine_rejects_wrapping_counts_and_non_finite_inputs(over):
    """alm_add_turbine applies the same count and finiteness checks (the GPU
    is needed only to create the lattice the rotor is added to)."""
    L = lbm.load()
    g = lbm.Lattice.create(64, 40, 40)
    hub = over.pop("hub", None)
    d, keep = _static_desc(**over)
    if hub is not None:
        for a in range(3):
            d.hub[a] = hub[a]
    tid = ctypes.c_int()
    assert L.alm_add_turbine(g._h, ctypes.byref(d), ctypes.byref(tid)) == INVALID_ARG
    g.destroy()
