"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: FP32 collision arithmetic on FP32 offsets f - w gives velocity
errors of a few 1e-9 per step; the bound max|du| <= 1e-6 lattice units on
laminar cases leaves room for a few hundred steps of accumulation.  PDFs are
compared element by element after one step to 2e-7 (absolute, f ~ 0.3).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2402_13171_gb300 import inputs as I
from cases import gpu_lattice, max_du, setup_pair

pytestmark = pytest.mark.gpu

DU_TOL = 1e-6
F_TOL = 2e-7


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_13171_gb300 import build
    build.build()
    O.build()


def test_taylor_green_32_cubed_200_steps():
    """3-D Taylor-Green vortex, 32^3, u0 = 0.05, nu = 0.01, 200 steps, cumulant."""
    dom = dict(nx=32, ny=32, nz=32, nu=0.01)
    rho, u = I.taylor_green_3d(32, 0.05)
    g, s = setup_pair(dom, rho=rho, u=u)
    g.step(200)
    s.step(200)
    du = max_du(g, s)
    print(f"TGV 32^3 200 steps: max|du| = {du:.3e}")
    assert du <= DU_TOL
    # kinetic energy follows the oracle's
    rg, ug = g.moments()
    ro, uo = s.moments()
    Eg = 0.5 * np.sum(rg * (ug ** 2).sum(0))
    Eo = 0.5 * np.sum(ro * (uo ** 2).sum(0))
    # |dE|/E <~ 2 max|du| / u0 = 4e-5 at the velocity bound
    assert Eg == pytest.approx(Eo, rel=4e-5)


def _gpu_energy(g):
    rho, u = g.moments()
    return 0.5 * float(np.sum(rho * (u ** 2).sum(0)))


@pytest.mark.parametrize("case", ["2d_exact", "3d_stokes"])
def test_taylor_green_decay_on_gpu_matches_analytic(case):
    """The 32^3 Taylor-Green configuration on the GPU against the analytic
    kinetic-energy decay: the z-invariant vortex is an exact Navier-Stokes
    solution, E ~ exp(-4 nu k^2 t); the 3-D vortex at small amplitude decays as
    its Stokes limit, E ~ exp(-6 nu k^2 t).  The rate between steps 20 and 200
    (after the start-up transient of an equilibrium initial state) gives the
    viscosity, within the lattice error the oracle's pins bound at this size."""
    n, nu, steps = 32, 0.01, 200
    if case == "2d_exact":
        dom = dict(nx=n, ny=n, nz=1, nu=nu)
        rho, u = I.taylor_green_2d(n, 0.05)
        rate_k2 = 4.0
    else:
        dom = dict(nx=n, ny=n, nz=n, nu=nu)
        rho, u = I.taylor_green_3d(n, 0.005)
        rate_k2 = 6.0
    g = gpu_lattice(dom)
    g.init_fields(rho, u, None)
    g.step(steps // 10)
    E1 = _gpu_energy(g)
    g.step(steps - steps // 10)
    E2 = _gpu_energy(g)
    k = 2 * math.pi / n
    nu_seen = -math.log(E2 / E1) / (steps - steps // 10) / (rate_k2 * k * k)
    print(f"TGV {case}: nu from the energy decay {nu_seen:.6f} (nu = {nu})")
    assert nu_seen == pytest.approx(nu, rel=1.5e-2)
    g.destroy()


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
@pytest.mark.parametrize("shape", [(37, 19, 11), (5, 4, 3), (1, 1, 1), (130, 3, 2)])
def test_one_step_pdfs_random_state(coll, shape):
    """Seeded near-equilibrium state on ragged periodic lattices (tails of the
    128-wide tiles, single cells): every post-collision PDF after one step."""
    nx, ny, nz = shape
    dom = dict(nx=nx, ny=ny, nz=nz, collision=coll, nu=0.02, smag_c=0.17, body_force=(1e-5, -2e-5, 3e-6))
    rho, u, fneq = I.random_state(nx, ny, nz, seed=101 + nx)
    g, s = setup_pair(dom, rho=rho, u=u, fneq=fneq)
    np.testing.assert_allclose(g.pdfs(), s.f, atol=F_TOL, rtol=0)
    g.step(1)
    s.step(1)
    np.testing.assert_allclose(g.pdfs(), s.f, atol=F_TOL, rtol=0)
    g.step(4)
    s.step(4)
    assert max_du(g, s) <= DU_TOL


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
def test_bounce_back_poiseuille(coll):
    dom = dict(nx=3, ny=16, nz=2, collision=coll, nu=0.1, bc=("periodic", "noslip", "periodic"),
               body_force=(1e-6, 0, 0))
    g, s = setup_pair(dom)
    g.step(300)
    s.step(300)
    assert max_du(g, s) <= DU_TOL
    dom2 = dict(nx=7, ny=9, nz=6, collision=coll, nu=0.05, bc=("noslip", "noslip", "noslip"),
                body_force=(1e-5, 5e-6, -3e-6))
    rho, u, fneq = I.random_state(7, 9, 6, seed=7)
    g, s = setup_pair(dom2, rho=rho, u=u, fneq=fneq)
    g.step(1)
    s.step(1)
    np.testing.assert_allclose(g.pdfs(), s.f, atol=F_TOL, rtol=0)
    g.step(20)
    s.step(20)
    assert max_du(g, s) <= DU_TOL


@pytest.mark.parametrize("bc", [("inout", "periodic", "freeslip"), ("freeslip", "noslip", "freeslip"),
                                ("inout", "freeslip", "noslip")])
def test_free_slip_walls(bc):
    """Specular walls (and their corners with inlet, outlet and no-slip faces):
    one-step PDFs and a short run against the oracle."""
    dom = dict(nx=23, ny=9, nz=11, nu=0.02, bc=bc, u_ref=(0.04, 0.01, 0.0), noise_rel=0.01, seed=77,
               body_force=(2e-6, 0, -1e-6))
    rho, u, fneq = I.random_state(23, 9, 11, seed=5, u_mean=(0.04, 0.01, 0.0))
    g, s = setup_pair(dom, rho=rho, u=u, fneq=fneq, inflow=bc[0] == "inout")
    g.step(1)
    s.step(1)
    np.testing.assert_allclose(g.pdfs(), s.f, atol=F_TOL, rtol=0)
    g.step(30)
    s.step(30)
    assert max_du(g, s) <= DU_TOL


def test_inlet_outlet_noise():
    dom = dict(nx=40, ny=12, nz=9, nu=0.01, bc=("inout", "periodic", "periodic"), u_ref=(0.05, 0.0, 0.0),
               noise_rel=0.01, seed=12345)
    g, s = setup_pair(dom, inflow=True)
    g.step(1)
    s.step(1)
    np.testing.assert_allclose(g.pdfs(), s.f, atol=F_TOL, rtol=0)
    g.step(60)
    s.step(60)
    assert max_du(g, s) <= DU_TOL


def small_rotor_case(collision="cumulant", kernel="gauss", tip_loss=False):
    dom, turb = I.single_turbine_case(64, 40, 40, diameter=16.0, elements_per_blade=8, seed=777, kernel=kernel,
                                      tip_loss=tip_loss)
    dom["collision"] = collision
    return dom, turb


@pytest.mark.parametrize("coll,kernel,tip_loss", [("cumulant", "gauss", False), ("srt_smag", "gauss", False),
                                                  ("cumulant", "roma", False), ("cumulant", "gauss", True)])
def test_rotor_short_horizon(coll, kernel, tip_loss):
    """Actuator line + inlet/outlet + noise on a scaled-down single-rotor case:
    flow, element forces and FP64 rotor loads stay with the oracle, for both
    regularisation kernels and with Glauert's tip-loss factor."""
    dom, turb = small_rotor_case(coll, kernel, tip_loss)
    g, s = setup_pair(dom, [turb], inflow=True)
    for n in (1, 10, 50):
        g.step(n - s.step_count)
        s.step(n - s.step_count)
        du = max_du(g, s)
        th, tq, ef, ep = g.loads(0, elements=True)
        print(f"{coll}/{kernel}/tip_loss={tip_loss} step {n}: max|du| {du:.2e}  thrust {th:.6e} vs {s.loads[0, 0]:.6e}")
        assert du <= DU_TOL
        np.testing.assert_allclose(ep, s.elem_pos, atol=2e-5)
        # element forces scale with |u_rel|^2: relative error ~ 2 max|du| / |u_rel| <= 2e-6 / 0.05
        np.testing.assert_allclose(ef, s.elem_force, atol=1e-7 + 5e-5 * np.abs(s.elem_force).max())
        assert th == pytest.approx(s.loads[0, 0], rel=5e-5)
        assert tq == pytest.approx(s.loads[0, 1], rel=5e-5)


@pytest.mark.parametrize("kernel", ["gauss", "roma"])
def test_rotor_force_sum_matches_blade_forces(kernel):
    """One step of momentum change equals minus the applied blade forces.

    The background is a uniform flow, whose cells all round alike in FP32; the
    same lattice without the rotor is stepped beside it, so that every cell
    outside the force support (bitwise the same in both) cancels and only the
    spread force remains."""
    dom, turb = small_rotor_case(kernel=kernel)
    dom["bc"] = ("periodic", "periodic", "periodic")
    u0 = np.stack([np.full((40, 40, 64), 0.05), np.zeros((40, 40, 64)), np.zeros((40, 40, 64))])
    g, s = setup_pair(dom, [turb], u=u0)
    g_free = gpu_lattice(dom)
    g_free.init_fields(None, u0, None)
    C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], dtype=np.float64)
    j0, j0_free = (np.einsum("qa,qzyx->a", C, L.pdfs()) for L in (g, g_free))
    _, _, ef0, _ = g.loads(0, elements=True)  # forces of step 0
    g.step(1)
    g_free.step(1)
    j1, j1_free = (np.einsum("qa,qzyx->a", C, L.pdfs()) for L in (g, g_free))
    dj = (j1 - j0) - (j1_free - j0_free)
    # ~2.5e4 cells in the force support, each rounding its momentum at ~1e-9
    np.testing.assert_allclose(dj, -ef0.astype(np.float64).sum(0), rtol=2e-6, atol=1e-7)
    g_free.destroy()


@pytest.mark.parametrize("kernel,tile", [("gauss", (32, 4, 1)), ("roma", (32, 4, 1)), ("gauss", (32, 8, 1))])
def test_full_size_single_turbine_sampled(kernel, tile):
    """256x128x128 single-rotor workload in the launch configurations the
    benchmark's tuner picks (32x4x1, 32x8x1): one step from a seeded state,
    checked at sampled cells (rotor box, inlet, outlet, bulk) and on every
    element force, against the oracle's per-cell update."""
    dom, turb = I.single_turbine_case(kernel=kernel)
    nx, ny, nz = dom["nx"], dom["ny"], dom["nz"]
    rho, u, fneq = I.random_state(nx, ny, nz, seed=4242, u_mean=(0.05, 0, 0), du=0.005, drho=0.002, fneq_amp=2e-4)
    g, s = setup_pair(dom, [turb], rho=rho, u=u, fneq=fneq, inflow=True, tile=tile)
    assert g.tile()[:3] == tile
    f0 = s.f.copy()
    # oracle: element forces of step 0 and the spread force at sampled cells
    pos, fb, alpha, loads = s.alm_forces(f0, np.zeros((3, nz, ny, nx)), 0)
    th, tq, ef, ep = g.loads(0, elements=True)
    np.testing.assert_allclose(ep, pos, atol=2e-5)
    np.testing.assert_allclose(ef, fb, atol=1e-5 * np.abs(fb).max())
    assert th == pytest.approx(loads[0], rel=1e-5)
    g.step(1)
    fg = g.pdfs()
    rng = np.random.default_rng(9)
    cells = [(0, 5, 7), (255, 127, 0), (64, 64, 64), (60, 50, 70), (70, 80, 48), (1, 0, 127), (254, 64, 3)]
    cells += [tuple(int(v) for v in c) for c in rng.integers([52, 42, 42], [76, 86, 86], (12, 3))]
    cells += [tuple(int(v) for v in c) for c in rng.integers([0, 0, 0], [256, 128, 128], (12, 3))]
    # cells nearest to every tenth element: inside even the 3-cell Roma support
    cells += [tuple(int(v) for v in np.round(p)) for p in pos[::10]]
    eps = turb["epsilon"]
    for (x, y, z) in cells:
        F = O.spread_at(pos, fb, eps, x, y, z, kernel=kernel)
        ref = s.update_cell(f0, F, 0, x, y, z)
        np.testing.assert_allclose(fg[:, z, y, x], ref, atol=F_TOL, rtol=0, err_msg=str((x, y, z)))


@pytest.mark.parametrize("tile", [(128, 1), (64, 2), (256, 1), (96, 1), (32, 8), (32, 4, 4), (32, 2, 7), (64, 2, 64),
                                  (32, 4, 2), (64, 1, 2)])
def test_tile_shapes_agree(tile):
    """Every CTA shape and marching depth (rotor tiles merged over up to 3
    single-plane z-blocks, or one z-block of tile_z planes) steps bitwise like
    the default."""
    dom, turb = small_rotor_case()
    ga, _ = setup_pair(dom, [turb], inflow=True)
    gb, _ = setup_pair(dom, [turb], inflow=True, tile=tile)
    ga.step(7)
    gb.step(7)
    np.testing.assert_array_equal(ga.pdfs(), gb.pdfs())
    assert ga.loads(0) == gb.loads(0)


@pytest.mark.parametrize("bc", [("periodic", "periodic", "periodic"), ("inout", "periodic", "freeslip"),
                                ("noslip", "noslip", "periodic"), ("freeslip", "freeslip", "noslip")])
@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_staged_rows_match_direct_loads(bc, storage):
    """Rows staged in shared memory by persistent CTAs give bitwise the same
    step as direct loads: wrap lanes, a ragged last segment (nx = 104 with
    64-wide segments), inlet/outlet and wall faces, a rotor, diagnostics."""
    nx = 104
    dom, turb = I.single_turbine_case(nx, 40, 40, diameter=16.0, elements_per_blade=8, seed=91)
    dom["bc"] = bc
    rho, u, fneq = I.random_state(nx, 40, 40, seed=8, u_mean=(0.04, 0.0, 0.0), du=0.01)
    ga, _ = setup_pair(dom, [turb], rho=rho, u=u, fneq=fneq, inflow=bc[0] == "inout", storage=storage, diag_every=3)
    gb, _ = setup_pair(dom, [turb], rho=rho, u=u, fneq=fneq, inflow=bc[0] == "inout", storage=storage, diag_every=3,
                       tile=(64, 1, 1, 1))
    assert gb.tile() == (64, 1, 1, 1)
    ga.step(7)
    gb.step(7)
    np.testing.assert_array_equal(ga.pdfs(), gb.pdfs())
    assert ga.loads(0) == gb.loads(0)
    da, _ = ga.diagnostics()
    db, _ = gb.diagnostics()
    np.testing.assert_allclose(da, db, rtol=0, atol=1e-9)


def test_staged_batch_matches_direct():
    from paper_2402_13171_gb300 import lbm
    cases = [I.single_turbine_case(64, 40, 40, diameter=16.0, elements_per_blade=8, seed=s) for s in (1, 2)]
    cases.append(I.single_turbine_case(96, 48, 44, diameter=20.0, elements_per_blade=6, seed=3))
    runs = []
    for tile in ((32, 4, 1, 0), (128, 1, 1, 1)):
        cfgs = [dict(nx=d["nx"], ny=d["ny"], nz=d["nz"], nu=d["nu"], bc=d["bc"], seed=d["seed"], tile=tile,
                     diag_every=4) for d, _ in cases]
        lat = lbm.batch_create(cfgs)
        for L, (d, t) in zip(lat, cases):
            L.set_inflow(u_ref=d["u_ref"], noise_rel=d["noise_rel"])
            L.add_turbine(**t)
        lat[0].step(9)
        runs.append([(L.pdfs(), L.loads(0), L.diagnostics()[0]) for L in lat])
    for (fa, la, da), (fb, lb, db) in zip(*runs):
        np.testing.assert_array_equal(fa, fb)
        assert la == lb
        np.testing.assert_allclose(da, db, rtol=0, atol=1e-9)


def test_two_rotors_of_many_elements():
    """Two rotors of 3 x 40 elements on one lattice, one of them yawed: the
    actuator-line launch runs 8 CTAs of 32 elements (the second rotor starting
    inside the fourth), the last adding up the loads.  Flow, element positions
    and forces and both rotors' loads follow the oracle, and the staged kernel
    (its own element culling per row segment) steps bit for bit like the direct
    one."""
    nx = 112
    dom, t1 = I.single_turbine_case(nx, 40, 40, diameter=16.0, elements_per_blade=40, seed=93, hub=(28.0, 20.0, 20.0))
    t2 = I.single_turbine(nx, 40, 40, diameter=16.0, elements_per_blade=40, hub=(72.0, 20.5, 19.5), yaw=0.12,
                          tsr=5.0)
    rho, u, fneq = I.random_state(nx, 40, 40, seed=9, u_mean=(0.04, 0.0, 0.0), du=0.01)
    ga, s = setup_pair(dom, [t1, t2], rho=rho, u=u, fneq=fneq, inflow=True, diag_every=3)
    gb, _ = setup_pair(dom, [t1, t2], rho=rho, u=u, fneq=fneq, inflow=True, diag_every=3, tile=(64, 1, 1, 1))
    assert ga.launches_per_step() == 3 and gb.launches_per_step() == 2
    ga.step(7)
    gb.step(7)
    s.step(7)
    _rotor_checks(ga, s, [t1, t2], "two rotors")
    np.testing.assert_array_equal(ga.pdfs(), gb.pdfs())
    for t in (0, 1):
        tha, tqa, efa, epa = ga.loads(t, elements=True)
        thb, tqb, efb, epb = gb.loads(t, elements=True)
        assert (tha, tqa) == (thb, tqb)
        np.testing.assert_array_equal(efa, efb)
        np.testing.assert_array_equal(epa, epb)
    ga.destroy()
    gb.destroy()


def test_autotune_keeps_state_and_results(tmp_path):
    """The tuner times tile candidates on the live state and restores it: the
    run continues exactly as an untuned one."""
    import os
    dom, turb = small_rotor_case()
    ga, _ = setup_pair(dom, [turb], inflow=True)
    gb, _ = setup_pair(dom, [turb], inflow=True)
    ga.step(5)
    gb.step(5)
    cache = str(tmp_path / "tune_cache.txt")
    if os.path.exists(cache):
        os.remove(cache)
    tile, ms = gb.autotune(steps=3, cache=cache)
    assert ms > 0 and gb.tile() == tile
    assert gb.step_count() == 5
    ga.step(6)
    gb.step(6)
    np.testing.assert_array_equal(ga.pdfs(), gb.pdfs())
    assert ga.loads(0) == gb.loads(0)
    # a cache hit applies the stored tile without timing
    gc, _ = setup_pair(dom, [turb], inflow=True)
    tile2, ms2 = gc.autotune(steps=3, cache=cache)
    assert tile2 == tile and ms2 == pytest.approx(ms, rel=1e-6)


def test_graph_replay_equals_direct_launches():
    dom, turb = small_rotor_case()
    ga, _ = setup_pair(dom, [turb], inflow=True)
    gb, _ = setup_pair(dom, [turb], inflow=True)
    gb.set_profiling(True)
    ga.step(9)
    gb.step(9)
    np.testing.assert_array_equal(ga.pdfs(), gb.pdfs())
    ms, n = gb.kernel_time()
    assert n == 9 and ms > 0
    # a step is the rotor-tile launch, the actuator line and the rest; without a
    # rotor, one launch
    assert gb.launches_per_step() == 3
    g0 = gpu_lattice(dom)
    assert g0.launches_per_step() == 1
    g0.destroy()


def test_async_loads_match_synchronous_reads():
    """alm_get_loads_async enqueued after each of six steps, with no wait in
    between, gives every step's thrust and torque as the synchronising read
    does on an identical lattice."""
    import torch
    dom, turb = small_rotor_case()
    ga, _ = setup_pair(dom, [turb], inflow=True)
    gs, _ = setup_pair(dom, [turb], inflow=True)
    buf = torch.zeros((6, 2), dtype=torch.float64).pin_memory()
    ref = []
    for i in range(6):
        ga.step(1)
        ga.loads_async(buf[i])
        gs.step(1)
        ref.append(gs.loads(0))
    ga.sync()
    np.testing.assert_array_equal(buf.numpy(), np.array(ref))
    assert np.all(buf.numpy()[:, 0] > 0)
    ga.destroy()
    gs.destroy()


def test_loads_sink_matches_synchronous_reads():
    """With a zero-copy loads sink, the device writes each step's thrust and
    torque into the page-locked ring; they equal the synchronising read of an
    identical lattice, step after step.  A ring of the wrong shape is refused."""
    import torch
    dom, turb = small_rotor_case()
    ga, _ = setup_pair(dom, [turb], inflow=True)
    gs, _ = setup_pair(dom, [turb], inflow=True)
    ring = torch.zeros((3, 1, 2), dtype=torch.float64).pin_memory()
    ga.set_loads_sink(ring)
    for k in range(1, 9):
        ga.step(1)
        gs.step(1)
        ga.sync()
        if k >= 2:  # the loads of step k - 1 were evaluated during step k - 2, after the sink was set
            assert tuple(ring[(k - 1) % 3, 0].tolist()) == gs.loads(0), k
    with pytest.raises(ValueError):
        ga.set_loads_sink(torch.zeros((3, 2, 2), dtype=torch.float64).pin_memory())  # wrong rotor count
    ga.destroy()
    gs.destroy()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_checkpoint_resume_is_bitwise(storage):
    """A lattice with a rotor, inlet noise and diagnostics, checkpointed after
    11 steps (lbm_get_state) and restored into a lattice with another history:
    at step 17 PDFs, rotor loads and element forces are bit for bit those of
    the uninterrupted run, and the diagnostic sums equal to FP64 rounding."""
    dom, turb = small_rotor_case()
    ga, _ = setup_pair(dom, [turb], inflow=True, storage=storage, diag_every=4)
    ga.step(11)
    blob = ga.state()
    ga.step(6)
    gb, _ = setup_pair(dom, [turb], inflow=True, storage=storage, diag_every=4)
    gb.step(3)          # different history, then restore
    gb.set_state(blob)
    assert gb.step_count() == 11
    gb.step(6)
    np.testing.assert_array_equal(ga.pdfs(), gb.pdfs())
    tha, tqa, efa, epa = ga.loads(0, elements=True)
    thb, tqb, efb, epb = gb.loads(0, elements=True)
    assert (tha, tqa) == (thb, tqb)
    np.testing.assert_array_equal(efa, efb)
    np.testing.assert_array_equal(epa, epb)
    assert ga.diagnostics()[1] == gb.diagnostics()[1] == 16
    # the FP64 sums add per-CTA partials in arrival order: equal to rounding
    np.testing.assert_allclose(ga.diagnostics()[0], gb.diagnostics()[0], rtol=1e-12, atol=1e-12)
    # a state of another lattice shape or rotor set is refused
    gc = gpu_lattice(dict(dom, nx=dom["nx"] + 8))
    from paper_2402_13171_gb300 import lbm
    with pytest.raises(lbm.LbmError, match="invalid argument"):
        gc.set_state(blob)
    gc.destroy()


def test_checkpoint_resume_at_odd_step_and_in_a_batch():
    """The state taken at an odd step restores into a lattice at an even step
    (the live array changes side), and a batch member restores from a state
    taken alone."""
    from paper_2402_13171_gb300 import lbm
    dom, turb = small_rotor_case()
    ga, _ = setup_pair(dom, [turb], inflow=True)
    ga.step(7)
    blob = ga.state()
    ga.step(5)
    d2 = dict(nx=33, ny=17, nz=9, nu=0.02, body_force=(1e-5, 0, 0))
    cfgs = [dict(nx=dom["nx"], ny=dom["ny"], nz=dom["nz"], nu=dom["nu"], bc=dom["bc"], seed=dom["seed"]),
            dict(nx=33, ny=17, nz=9, nu=0.02, body_force=(1e-5, 0, 0))]
    lat = lbm.batch_create(cfgs)
    lat[0].set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
    lat[0].add_turbine(**turb)
    rho, u, fneq = I.random_state(33, 17, 9, seed=3)
    lat[1].init_fields(rho, u, fneq)
    g1, _ = setup_pair(d2, rho=rho, u=u, fneq=fneq)
    g1.step(7)
    lat[0].step(2)
    lat[1].set_state(g1.state())       # both members now at step 7
    lat[0].set_state(blob)
    lat[0].step(5)
    g1.step(5)
    np.testing.assert_array_equal(lat[0].pdfs(), ga.pdfs())
    assert lat[0].loads(0) == ga.loads(0)
    np.testing.assert_array_equal(lat[1].pdfs(), g1.pdfs())


def test_pdf_restore_without_force_box_stays_close():
    """lbm_set_pdfs + lbm_set_step restore the populations and step but not
    the lagged rotor force, so a rotor run resumed that way departs from the
    original by a small amount near the rotor; a lattice without rotors
    resumes bit for bit."""
    dom, turb = small_rotor_case()
    ga, _ = setup_pair(dom, [turb], inflow=True)
    ga.step(11)
    f = ga.pdfs()
    n = ga.step_count()
    ga.step(6)
    gb, _ = setup_pair(dom, [turb], inflow=True)
    gb.step(3)          # different history, then restore
    gb.set_pdfs(f)
    gb.set_step(n)
    gb.step(6)
    fa, fb = ga.pdfs(), gb.pdfs()
    assert np.abs(fa - fb).max() < 1e-4
    dom2 = dict(nx=20, ny=10, nz=6, nu=0.02, bc=("inout", "periodic", "periodic"), u_ref=(0.04, 0, 0),
                noise_rel=0.01, seed=5)
    ha, _ = setup_pair(dom2, inflow=True)
    ha.step(13)
    f = ha.pdfs()
    ha.step(5)
    hb, _ = setup_pair(dom2, inflow=True)
    hb.set_pdfs(f)
    hb.set_step(13)
    hb.step(5)
    np.testing.assert_array_equal(ha.pdfs(), hb.pdfs())


def test_probe_matches_moments():
    dom, turb = small_rotor_case()
    g, _ = setup_pair(dom, [turb], inflow=True)
    g.step(9)
    rho, u = g.moments()
    rng = np.random.default_rng(4)
    x, y, z = rng.integers(0, 64, 50), rng.integers(0, 40, 50), rng.integers(0, 40, 50)
    x[:3], y[:3], z[:3] = 16, 20, 20  # hub: inside the rotor force box
    pr, pu = g.probe(x, y, z)
    np.testing.assert_array_equal(pr, rho[z, y, x])
    np.testing.assert_array_equal(pu, u[:, z, y, x].T)


def test_diagnostics_fp64_sums():
    """The fused FP64 sums equal the sums of the lattice's own PDFs (mass as
    the sum of the offsets f - w)."""
    dom = dict(nx=33, ny=17, nz=9, nu=0.02, body_force=(1e-5, 0, 0))
    rho, u, fneq = I.random_state(33, 17, 9, seed=3)
    g, s = setup_pair(dom, rho=rho, u=u, fneq=fneq, diag_every=5)
    g.step(11)  # diagnostic steps 0, 5, 10
    mm, at = g.diagnostics()
    assert at == 10
    f = g.pdfs()
    # sums of the offsets: mass - N, momentum
    assert mm[0] == pytest.approx((f.sum() - f[0].size), abs=1e-6)
    np.testing.assert_allclose(mm[1:], np.einsum("qa,qzyx->a", C27, f), atol=1e-6)


C27 = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], dtype=np.float64)


@pytest.mark.parametrize("case", ["periodic_body_force", "rotor_inlet_outlet", "log_law_farm"])
def test_diagnostics_match_oracle(case):
    """The fused FP64 mass and momentum of the last diagnostic step against the
    oracle's state after the same steps: a periodic lattice with a body force
    (mass conserved, momentum grows by F per cell and step), the rotor case
    with inlet noise and outlet, and the log-law farm with free-slip walls
    (neither conserves momentum).  Tolerance: each cell's offsets stay within
    the 2e-7 PDF parity bound, whose errors do not share a sign, so the sums
    over N cells stay within 27 * 2e-7 * sqrt(N) (2e-3 at N = 1e5)."""
    if case == "periodic_body_force":
        dom = dict(nx=33, ny=17, nz=9, nu=0.02, body_force=(1e-5, 0, -3e-6))
        rho, u, fneq = I.random_state(33, 17, 9, seed=3)
        g, s = setup_pair(dom, rho=rho, u=u, fneq=fneq, diag_every=5)
    elif case == "rotor_inlet_outlet":
        dom, turb = small_rotor_case()
        g, s = setup_pair(dom, [turb], inflow=True, diag_every=5)
    else:
        dom, turbs = I.small_farm_case(nx=64, ny=32, nz=28, diameter=8.0, elements_per_blade=4, x_hubs=(14.0, 40.0))
        g, s = setup_pair(dom, turbs, inflow=True, diag_every=5)
    g.step(11)
    s.step(11)
    mm, at = g.diagnostics()
    assert at == 10
    N = s.f[0].size
    mass_o = s.f.sum() - N
    mom_o = np.einsum("qa,qzyx->a", C27, s.f)
    tol = 27 * 2e-7 * math.sqrt(N)
    assert mm[0] == pytest.approx(mass_o, abs=tol)
    np.testing.assert_allclose(mm[1:], mom_o, rtol=0, atol=tol)
    if case == "periodic_body_force":
        assert mm[0] == pytest.approx(s.f.sum() - N, abs=1e-6 * N ** 0.5)
    else:
        assert abs(mom_o[0]) > 10 * tol   # momentum carried by the inflow: the check is not vacuous


def test_batch_equals_separate_runs():
    """Three lattices in one batch (a Gaussian rotor; a Roma rotor with tip
    loss; no rotor) step bitwise as they do alone."""
    from paper_2402_13171_gb300 import lbm
    dom1, t1 = I.single_turbine_case(64, 40, 40, diameter=16.0, elements_per_blade=8, seed=1)
    dom2, t2 = I.single_turbine_case(72, 48, 44, diameter=20.0, elements_per_blade=6, seed=2, tsr=4.0, u_inf=0.04,
                                     kernel="roma", tip_loss=True)
    dom3 = dict(nx=33, ny=17, nz=9, nu=0.02, body_force=(1e-5, 0, 0))
    cfgs = []
    for d in (dom1, dom2, dom3):
        cfgs.append(dict(nx=d["nx"], ny=d["ny"], nz=d["nz"], collision="cumulant", nu=d["nu"],
                         bc=d.get("bc", ("periodic",) * 3), body_force=d.get("body_force", (0, 0, 0)),
                         seed=d.get("seed", 0)))
    lat = lbm.batch_create(cfgs)
    singles = []
    for d, t, L in ((dom1, t1, lat[0]), (dom2, t2, lat[1]), (dom3, None, lat[2])):
        gs, _ = setup_pair(d, [t] if t else [], inflow="u_ref" in d)
        singles.append(gs)
        if "u_ref" in d:
            L.set_inflow(u_ref=d["u_ref"], noise_rel=d["noise_rel"])
        if t:
            L.add_turbine(**t)
        if "u_ref" not in d:
            L.init_fields()
    lat[0].step(12)
    for gs in singles:
        gs.step(12)
    for L, gs in zip(lat, singles):
        np.testing.assert_array_equal(L.pdfs(), gs.pdfs())
    assert lat[0].loads(0) == singles[0].loads(0)
    assert lat[1].loads(0) == singles[1].loads(0)


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_sixteen_bit_storage_tracks_fp32(storage):
    dom = dict(nx=32, ny=32, nz=32, nu=0.01)
    rho, u = I.taylor_green_3d(32, 0.05)
    g32, s = setup_pair(dom, rho=rho, u=u)
    g16, _ = setup_pair(dom, rho=rho, u=u, storage=storage)
    g32.step(100)
    g16.step(100)
    s.step(100)
    _, u32 = g32.moments()
    _, u16 = g16.moments()
    _, uo = s.moments()
    err = np.abs(u16 - uo).max()
    print(f"{storage}: max|du| vs oracle {err:.3e}, fp32 {np.abs(u32 - uo).max():.3e}")
    # 8-bit (bf16) / 11-bit (fp16) mantissas on offsets of ~0.05: per-step rounding 2e-4 / 2.5e-5
    assert err < (1e-3 if storage == "bf16" else 1e-4)


def _rotor_checks(g, s, turbs, tag):
    du = max_du(g, s)
    print(f"{tag} step {s.step_count}: max|du| {du:.2e}")
    assert du <= DU_TOL
    off = 0
    for t_i, t in enumerate(turbs):
        ne = t["n_blades"] * t["n_elements"]
        th, tq, ef, ep = g.loads(t_i, elements=True)
        np.testing.assert_allclose(ep, s.elem_pos[off:off + ne], atol=2e-5)
        fo = s.elem_force[off:off + ne]
        np.testing.assert_allclose(ef, fo, atol=1e-7 + 5e-5 * np.abs(fo).max())
        assert th == pytest.approx(s.loads[t_i, 0], rel=5e-5)
        assert tq == pytest.approx(s.loads[t_i, 1], rel=5e-5)
        off += ne


@pytest.mark.parametrize("coll,kernel", [("cumulant", "gauss"), ("srt_smag", "gauss"), ("cumulant", "roma")])
def test_yawed_twisted_pitched_rotor_on_unequal_polars(coll, kernel):
    """A rotor yawed by 7 degrees, with a twist table, a collective pitch and a
    start angle, on polars tabulated at unequal angles (the table search of the
    non-uniform branch): flow, element positions and forces and FP64 loads
    stay with the oracle over 50 steps."""
    dom, turb = I.yawed_twisted_rotor(kernel=kernel)
    dom["collision"] = coll
    g, s = setup_pair(dom, [turb], inflow=True)
    for n in (1, 10, 50):
        g.step(n - s.step_count)
        s.step(n - s.step_count)
        _rotor_checks(g, s, [turb], f"yawed {coll}/{kernel}")


def test_log_law_farm_two_yawed_rotors():
    """A scaled-down farm: log-law inflow with noise, free-slip bottom and top,
    periodic y, zero-gradient outlet and two yawed rotors in a row, the second
    in the wake of the first.  The initial state is the log profile on both
    sides; one step matches PDF for PDF, then the flow and every rotor's loads
    stay with the oracle over 40 steps."""
    dom, turbs = I.small_farm_case()
    g, s = setup_pair(dom, turbs, inflow=True)
    _, u0 = g.moments()
    prof = I.log_law_profile(dom["nz"], dom["u_ref"][0], dom["z0"], dom["z_ref"])
    np.testing.assert_allclose(u0[0, :, 5, 5], prof, atol=1e-8)
    g.step(1)
    s.step(1)
    np.testing.assert_allclose(g.pdfs(), s.f, atol=F_TOL, rtol=0)
    for n in (10, 40):
        g.step(n - s.step_count)
        s.step(n - s.step_count)
        _rotor_checks(g, s, turbs, "log-law farm")
