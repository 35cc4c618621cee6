"""Host-side argument checks of the C ABI, which run before any CUDA call:
lattice sizes (including the 32-bit plane-offset limit 27 N < 2^31), boundary
codes, viscosity, tiles, and batches whose members disagree."""
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
