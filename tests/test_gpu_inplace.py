"""The in-place (AA) scheme against the two-array pull scheme.

After every even number of steps the single AA array holds exactly the pull
scheme's state, so the two are compared bitwise, on periodic and no-slip
lattices, both collisions and 16-bit storage, through graph replays and single
launches; with the rotor workload's inlet noise, outlet and actuator line; with
free-slip walls; on a two-rotor log-law lattice; odd step counts refuse state
access; the PDF memory is halved; and the oracle confirms the pull scheme these
are compared with."""
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


def _rotor_pair(dom, turbs, storage="fp32", diag_every=0):
    kw = dict(collision=dom.get("collision", "cumulant"), nu=dom["nu"], smag_c=dom.get("smag_c", 0.1), storage=storage,
              bc=dom["bc"], seed=dom["seed"], diag_every=diag_every)
    out = []
    for inplace in (False, True):
        g = lbm.Lattice.create(dom["nx"], dom["ny"], dom["nz"], inplace=inplace, **kw)
        g.set_inflow(u_ref=dom["u_ref"], kind=dom.get("inflow_kind", 0), z0=dom.get("z0", 0.1),
                     z_ref=dom.get("z_ref", 1.0), noise_rel=dom["noise_rel"])
        for t in turbs:
            g.add_turbine(**t)
        out.append(g)
    return out


def _same_run(g2, ga, n_turb, counts=(10, 1, 1, 2, 8, 6)):
    for n in counts:   # graph replays of 8 and 2, single odd and even launches
        g2.step(n)
        ga.step(n)
        if ga.step_count() % 2:
            continue
        np.testing.assert_array_equal(ga.pdfs(), g2.pdfs())
        for t in range(n_turb):
            th2, tq2, ef2, ep2 = g2.loads(t, elements=True)
            tha, tqa, efa, epa = ga.loads(t, elements=True)
            assert (tha, tqa) == (th2, tq2)
            np.testing.assert_array_equal(efa, ef2)
            np.testing.assert_array_equal(epa, ep2)


@pytest.mark.parametrize("collision,storage,kernel", [("cumulant", "fp32", "gauss"), ("cumulant", "bf16", "gauss"),
                                                      ("srt_smag", "fp32", "roma")])
def test_inplace_rotor_inlet_outlet_equals_two_arrays_bitwise(collision, storage, kernel):
    """The rotor workload's scaled-down case on one array: velocity inlet with
    noise, zero-gradient outlet, the actuator line (its sampling reads the array
    in the layout each step leaves) -- bit for bit the two-array run at every
    even step, loads and element forces included, with diagnostics."""
    dom, turb = I.single_turbine_case(64, 40, 40, diameter=16.0, elements_per_blade=8, seed=777, kernel=kernel)
    dom["collision"] = collision
    g2, ga = _rotor_pair(dom, [turb], storage, diag_every=4)
    assert ga.launches_per_step() == 3  # rotor tiles, actuator line, the rest
    _same_run(g2, ga, 1)
    d2, s2 = g2.diagnostics()
    da, sa = ga.diagnostics()
    assert s2 == sa
    np.testing.assert_allclose(da, d2, rtol=0, atol=1e-9)
    g2.destroy()
    ga.destroy()


@pytest.mark.parametrize("bc", [("inout", "periodic", "freeslip"), ("freeslip", "noslip", "freeslip"),
                                ("inout", "freeslip", "noslip"), ("periodic", "freeslip", "periodic")])
def test_inplace_free_slip_and_inlet_faces_equal_two_arrays_bitwise(bc):
    """Free-slip faces and their corners with inlet, outlet and no-slip faces
    on one array: a slot a free-slip face reflects into has one reader, so the
    write-back into the slot read stays exact."""
    nx, ny, nz = 23, 9, 11
    kw = dict(nu=0.02, bc=bc, body_force=(2e-6, 0, -1e-6), seed=77)
    rho, u, fneq = I.random_state(nx, ny, nz, seed=5, u_mean=(0.04, 0.01, 0.0))
    out = []
    for inplace in (False, True):
        g = lbm.Lattice.create(nx, ny, nz, inplace=inplace, **kw)
        if bc[0] == "inout":
            g.set_inflow(u_ref=(0.04, 0.01, 0.0), noise_rel=0.01)
        g.init_fields(rho, u, fneq)
        out.append(g)
    g2, ga = out
    _same_run(g2, ga, 0)
    g2.destroy()
    ga.destroy()


def test_inplace_log_law_farm_equals_two_arrays_bitwise():
    """The scaled-down farm on one array: log-law inflow with noise, free-slip
    bottom and top, periodic y, two yawed rotors."""
    dom, turbs = I.small_farm_case()
    g2, ga = _rotor_pair(dom, turbs, diag_every=5)
    _same_run(g2, ga, 2, counts=(8, 2, 1, 1, 10))
    g2.destroy()
    ga.destroy()


def test_inplace_rotor_step_pair_matches_oracle_and_resumes_bitwise():
    """One step pair of the in-place rotor case against the FP64 oracle at the
    parity bound, and a checkpoint of the in-place lattice resumes bit for bit."""
    from cases import oracle_sim
    dom, turb = I.single_turbine_case(64, 40, 40, diameter=16.0, elements_per_blade=8, seed=777)
    _, ga = _rotor_pair(dom, [turb])
    s = oracle_sim(dom, [turb])
    s.init_fields()
    ga.step(2)
    s.step(2)
    assert max_du(ga, s) <= 1e-6
    th, tq = ga.loads(0)
    assert th == pytest.approx(s.loads[0, 0], rel=5e-5)
    blob = ga.state()
    ga.step(6)
    gb = _rotor_pair(dom, [turb])[1]
    gb.step(4)
    gb.set_state(blob)
    gb.step(6)
    np.testing.assert_array_equal(ga.pdfs(), gb.pdfs())
    assert ga.loads(0) == gb.loads(0)
    ga.destroy()
    gb.destroy()
