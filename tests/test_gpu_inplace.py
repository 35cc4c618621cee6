"""The in-place (AA) scheme against the two-array pull scheme.

After every even number of steps the single AA array holds exactly the pull
scheme's state, so the two are compared bitwise, on periodic and no-slip
lattices, both collisions and 16-bit storage, through graph replays and single
launches; odd step counts refuse state access; the PDF memory is halved; and
the oracle confirms the pull scheme these are compared with (one step)."""
import numpy as np
import pytest

import oracle as O
from paper_2402_13171_gb300 import inputs as I
from paper_2402_13171_gb300 import lbm
from cases import max_du, oracle_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_13171_gb300 import build
    build.build()
    O.build()


def _pair(shape, bc, collision="cumulant", storage="fp32", body=(0.0, 0.0, 0.0), diag_every=0, seed=3):
    nx, ny, nz = shape
    kw = dict(collision=collision, nu=0.02, smag_c=0.15, storage=storage, bc=bc, body_force=body,
              diag_every=diag_every)
    g2 = lbm.Lattice.create(nx, ny, nz, **kw)
    ga = lbm.Lattice.create(nx, ny, nz, inplace=True, **kw)
    rho, u, fneq = I.random_state(nx, ny, nz, seed=seed, u_mean=(0.03, -0.01, 0.02), du=0.01, drho=0.005)
    for g in (g2, ga):
        g.init_fields(rho, u, fneq)
    return g2, ga, (rho, u, fneq)


CASES = [((37, 19, 11), ("periodic",) * 3, (0.0, 0.0, 0.0)),
         ((40, 24, 18), ("noslip", "periodic", "noslip"), (1e-5, 0.0, 0.0)),
         ((24, 20, 16), ("noslip",) * 3, (0.0, 2e-5, -1e-5)),
         ((1, 9, 5), ("periodic", "noslip", "periodic"), (0.0, 0.0, 1e-5))]


@pytest.mark.parametrize("collision,storage", [("cumulant", "fp32"), ("srt_smag", "fp32"), ("cumulant", "bf16")])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_inplace_equals_two_arrays_bitwise(case, collision, storage):
    shape, bc, body = CASES[case]
    g2, ga, _ = _pair(shape, bc, collision, storage, body, diag_every=4)
    for n in (10, 1, 1, 2, 8):   # graph replays of 8 and 2, single odd/even launches
        g2.step(n)
        ga.step(n)
        if ga.step_count() % 2:
            with pytest.raises(lbm.LbmError, match="invalid state"):
                ga.pdfs()
            continue
        np.testing.assert_array_equal(ga.pdfs(), g2.pdfs())
        r2, u2 = g2.moments()
        ra, ua = ga.moments()
        np.testing.assert_array_equal(ua, u2)
    d2, s2 = g2.diagnostics()
    da, sa = ga.diagnostics()
    assert s2 == sa
    np.testing.assert_allclose(da, d2, rtol=0, atol=1e-9)
    assert ga.launches_per_step() == 1
    g2.destroy()
    ga.destroy()


def test_inplace_one_step_pair_matches_oracle():
    """Two steps of the in-place scheme against the FP64 oracle (no-slip
    channel with a body force): the same bound as the pull scheme's parity."""
    shape, bc, body = CASES[1]
    nx, ny, nz = shape
    _, ga, (rho, u, fneq) = _pair(shape, bc, body=body)
    dom = dict(nx=nx, ny=ny, nz=nz, collision="cumulant", nu=0.02, bc=bc, body_force=body)
    s = oracle_sim(dom)
    s.init_fields(rho, u, fneq)
    ga.step(2)
    s.step(2)
    assert max_du(ga, s) <= 1e-6
    ga.destroy()


def test_inplace_halves_pdf_memory_and_refuses_what_it_does_not_take():
    import torch
    nx, ny, nz = 64, 32, 32
    fbytes = 27 * nx * ny * nz * 4
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    g2 = lbm.Lattice.create(nx, ny, nz)
    m1 = torch.cuda.memory_allocated()
    ga = lbm.Lattice.create(nx, ny, nz, inplace=True)
    m2 = torch.cuda.memory_allocated()
    assert (m1 - m0) - (m2 - m1) >= fbytes            # one PDF array fewer
    dom, turb = I.single_turbine_case(64, 32, 32, diameter=8.0, elements_per_blade=4)
    with pytest.raises(lbm.LbmError, match="unsupported"):
        ga.add_turbine(**turb)
    with pytest.raises(lbm.LbmError, match="unsupported"):
        ga.set_tile(32, 4, 2)
    ga.step(3)
    with pytest.raises(lbm.LbmError, match="invalid state"):
        ga.moments()
    with pytest.raises(lbm.LbmError, match="invalid state"):
        ga.set_step(6)
    ga.step(1)
    ga.moments()                                      # even again: usable
    g2.destroy()
    ga.destroy()


def test_inplace_batch_equals_separate_two_array_runs():
    """Two in-place lattices of different sizes stepped as one batch match
    their two-array runs bitwise at even step counts."""
    shapes = [((20, 12, 9), ("periodic",) * 3), ((16, 10, 14), ("noslip", "periodic", "noslip"))]
    cfgs = [dict(nx=s[0], ny=s[1], nz=s[2], nu=0.02, bc=bc, body_force=(1e-5, 0.0, 0.0), inplace=True)
            for s, bc in shapes]
    lat = lbm.batch_create(cfgs)
    refs = []
    for i, (L, (s, bc)) in enumerate(zip(lat, shapes)):
        rho, u, fneq = I.random_state(*s, seed=40 + i, u_mean=(0.02, 0.0, 0.01), du=0.01, drho=0.005)
        L.init_fields(rho, u, fneq)
        g = lbm.Lattice.create(*s, nu=0.02, bc=bc, body_force=(1e-5, 0.0, 0.0))
        g.init_fields(rho, u, fneq)
        refs.append(g)
    lat[0].step(6)
    for L, g in zip(lat, refs):
        g.step(6)
        np.testing.assert_array_equal(L.pdfs(), g.pdfs())
        g.destroy()
