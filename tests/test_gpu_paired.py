"""The paired form of the bulk kernel against the one-cell form.

With 16-bit storage the bulk tiles (no cell on a no-slip or free-slip face)
take two cells of a row per thread: 32-bit loads and stores of bf16x2/f16x2
words and the collision (cumulant or BGK-Smagorinsky) on f32x2 instructions
across the pair.  Every operation rounds as the one-cell evaluation does, so PDFs, rotor
loads and element forces must agree bit for bit with the one-cell kernel
(``staged`` 2), on periodic and inlet/outlet lattices, ragged and degenerate
sizes (nx = 2: one pair on both x faces), several tile shapes, diagnostic steps
and a batch.  Where pairs do not apply (odd nx, FP32 storage) the library keeps
one cell per thread, and the 16-bit results are checked against the FP64 oracle
by the storage tests in test_gpu_parity.py.
"""
import numpy as np
import pytest

from paper_2402_13171_gb300 import inputs as I
from cases import gpu_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_13171_gb300 import build
    build.build()


def _run(dom, storage, tile, form, steps, state=None, turb=None, inflow=False, diag_every=0):
    g = gpu_lattice(dom, storage=storage, diag_every=diag_every, tile=tuple(tile) + (1, form))
    if inflow:
        g.set_inflow(u_ref=dom["u_ref"], noise_rel=dom.get("noise_rel", 0.0))
    if turb is not None:
        g.add_turbine(**turb)
    if state is not None:
        g.init_fields(*state)
    elif not inflow:
        g.init_fields(None, None, None)
    assert g.tile()[3] == form
    g.step(steps)
    out = {"pdfs": g.pdfs(), "diag": g.diagnostics()}
    if turb is not None:
        out["loads"] = g.loads(0, elements=True)
    g.destroy()
    return out


def _same(a, b):
    np.testing.assert_array_equal(a["pdfs"], b["pdfs"])
    if "loads" in a:
        tha, tqa, efa, epa = a["loads"]
        thb, tqb, efb, epb = b["loads"]
        assert (tha, tqa) == (thb, tqb)
        np.testing.assert_array_equal(efa, efb)
        np.testing.assert_array_equal(epa, epb)
    # the FP64 sums add per-thread partials in another grouping: equal to rounding
    np.testing.assert_allclose(a["diag"][0], b["diag"][0], rtol=1e-12, atol=1e-12)
    assert a["diag"][1] == b["diag"][1]


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("shape,tile", [((64, 12, 6), (32, 4)), ((70, 5, 3), (32, 4)), ((2, 3, 4), (32, 4)),
                                        ((130, 6, 5), (64, 2)), ((96, 4, 4), (128, 1)), ((66, 9, 3), (32, 8))])
def test_paired_bulk_matches_one_cell_periodic(coll, storage, shape, tile):
    nx, ny, nz = shape
    dom = dict(nx=nx, ny=ny, nz=nz, nu=0.02, body_force=(2e-6, -1e-6, 5e-7), collision=coll, smag_c=0.17)
    state = I.random_state(nx, ny, nz, seed=11)
    a = _run(dom, storage, tile, 0, 9, state=state, diag_every=4)
    b = _run(dom, storage, tile, 2, 9, state=state, diag_every=4)
    _same(a, b)


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("tile", [(32, 4), (64, 1)])
def test_paired_bulk_matches_one_cell_with_inlet_outlet_and_rotor(coll, storage, tile):
    """The rotor case: inlet ghost columns at x = 0 (the first cell of the first
    pair), the outlet's clamped source at x = nx - 1 (the second cell of the last
    pair), inflow noise, and a rotor whose sampling reads the pairs' stores."""
    dom, turb = I.single_turbine_case(64, 40, 40, diameter=16.0, elements_per_blade=8, seed=777)
    dom["collision"] = coll
    a = _run(dom, storage, tile, 0, 12, turb=turb, inflow=True, diag_every=5)
    b = _run(dom, storage, tile, 2, 12, turb=turb, inflow=True, diag_every=5)
    _same(a, b)


def test_paired_bulk_in_a_batch_with_an_odd_member_keeps_one_cell():
    """A batch whose lattices all have even nx pairs its bulk cells; one odd nx
    keeps the whole batch on one cell per thread.  Both agree with lattices
    stepped alone in the one-cell form."""
    from paper_2402_13171_gb300 import lbm
    shapes = [(40, 7, 5), (34, 9, 4)]
    for odd in (False, True):
        shp = shapes + ([(33, 6, 3)] if odd else [])
        cfgs = [dict(nx=n[0], ny=n[1], nz=n[2], nu=0.01 + 0.005 * i, storage="bf16") for i, n in enumerate(shp)]
        lat = lbm.batch_create(cfgs)
        states = [I.random_state(*n, seed=20 + i) for i, n in enumerate(shp)]
        for L, st in zip(lat, states):
            L.init_fields(*st)
        lat[0].step(7)  # steps every member
        lat[0].sync()
        for i, (L, n) in enumerate(zip(lat, shp)):
            dom = dict(nx=n[0], ny=n[1], nz=n[2], nu=0.01 + 0.005 * i)
            ref = _run(dom, "bf16", (32, 4), 2, 7, state=states[i])
            np.testing.assert_array_equal(L.pdfs(), ref["pdfs"])
        for L in lat:
            L.destroy()


def test_forms_where_pairs_do_not_apply():
    """FP32 storage and odd nx run one cell per thread whatever the form asks;
    the form is still reported as set, and the results do not depend on it."""
    for dom, storage in [(dict(nx=32, ny=8, nz=4, nu=0.02), "fp32"), (dict(nx=33, ny=8, nz=4, nu=0.02), "bf16")]:
        state = I.random_state(dom["nx"], dom["ny"], dom["nz"], seed=3)
        a = _run(dom, storage, (32, 4), 0, 5, state=state)
        b = _run(dom, storage, (32, 4), 2, 5, state=state)
        _same(a, b)


def _run_aa(dom, storage, tile, form, steps, state=None, turb=None, inflow=False, diag_every=0):
    """The in-place scheme (one PDF array) for `steps` steps, an even count."""
    from paper_2402_13171_gb300 import lbm
    g = lbm.Lattice.create(dom["nx"], dom["ny"], dom["nz"], collision=dom.get("collision", "cumulant"),
                           nu=dom.get("nu", 0.02), smag_c=dom.get("smag_c", 0.17), storage=storage,
                           bc=dom.get("bc", ("periodic",) * 3), body_force=dom.get("body_force", (0, 0, 0)),
                           seed=dom.get("seed", 0), diag_every=diag_every, tile=tuple(tile) + (1, form), inplace=True)
    if inflow:
        g.set_inflow(u_ref=dom["u_ref"], noise_rel=dom.get("noise_rel", 0.0))
    if turb is not None:
        g.add_turbine(**turb)
    if state is not None:
        g.init_fields(*state)
    elif not inflow:
        g.init_fields(None, None, None)
    out = []
    for n in steps:   # odd and even steps, graph replays and single launches
        g.step(n)
        if g.step_count() % 2 == 0:
            out.append(g.pdfs())
    loads = g.loads(0, elements=True) if turb is not None else None
    g.destroy()
    return out, loads


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("shape,tile,bc", [((64, 12, 6), (32, 4), ("periodic",) * 3),
                                           ((70, 5, 3), (32, 4), ("periodic",) * 3),
                                           ((2, 3, 4), (32, 4), ("periodic",) * 3),
                                           ((130, 6, 5), (64, 2), ("periodic",) * 3),
                                           ((40, 12, 10), (32, 4), ("periodic", "freeslip", "noslip"))])
def test_paired_inplace_matches_one_cell(coll, storage, shape, tile, bc):
    """The in-place scheme's paired form (odd steps on a pair's own words, even
    steps with half-word stores into the neighbours' words) against its
    one-cell form, bit for bit after every even step; on a lattice with wall
    faces the face tiles keep one cell per thread in a launch of their own."""
    nx, ny, nz = shape
    dom = dict(nx=nx, ny=ny, nz=nz, nu=0.02, body_force=(2e-6, -1e-6, 5e-7), collision=coll, bc=bc)
    state = I.random_state(nx, ny, nz, seed=13, u_mean=(0.03, -0.01, 0.02), du=0.01, drho=0.005)
    a, _ = _run_aa(dom, storage, tile, 0, (1, 1, 2, 8, 3, 1), state=state, diag_every=4)
    b, _ = _run_aa(dom, storage, tile, 2, (1, 1, 2, 8, 3, 1), state=state, diag_every=4)
    assert len(a) == len(b) == 4
    for fa, fb in zip(a, b):
        np.testing.assert_array_equal(fa, fb)


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
def test_paired_inplace_with_inlet_outlet_and_rotor(coll):
    """In place with the inlet ghosts (the x = 0 cell of the first pair), the
    outlet copies (the x = nx - 1 cell of the last pair), inflow noise and a
    rotor whose sampling reads the array in the layout each step leaves."""
    dom, turb = I.single_turbine_case(64, 40, 40, diameter=16.0, elements_per_blade=8, seed=777)
    dom["collision"] = coll
    a, la = _run_aa(dom, "bf16", (32, 4), 0, (1, 1, 2, 8), turb=turb, inflow=True, diag_every=5)
    b, lb = _run_aa(dom, "bf16", (32, 4), 2, (1, 1, 2, 8), turb=turb, inflow=True, diag_every=5)
    for fa, fb in zip(a, b):
        np.testing.assert_array_equal(fa, fb)
    assert la[:2] == lb[:2]
    np.testing.assert_array_equal(la[2], lb[2])
    np.testing.assert_array_equal(la[3], lb[3])


def test_paired_inplace_batch_matches_one_cell():
    """Two in-place BF16 lattices of different sizes (one with wall faces)
    stepped as one batch take the batch form of the paired in-place step;
    each member agrees bit for bit with its lattice run alone one cell per
    thread."""
    from paper_2402_13171_gb300 import lbm
    shapes = [((40, 7, 5), ("periodic",) * 3), ((34, 9, 6), ("periodic", "noslip", "freeslip"))]
    cfgs = [dict(nx=s[0], ny=s[1], nz=s[2], nu=0.01 + 0.005 * i, bc=bc, body_force=(1e-5, 0.0, 2e-6),
                 storage="bf16", inplace=True) for i, (s, bc) in enumerate(shapes)]
    lat = lbm.batch_create(cfgs)
    states = [I.random_state(*s, seed=60 + i, u_mean=(0.02, 0.0, 0.01), du=0.01, drho=0.005)
              for i, (s, _) in enumerate(shapes)]
    for L, st in zip(lat, states):
        L.init_fields(*st)
    lat[0].step(6)  # steps every member
    lat[0].sync()
    for i, (L, (s, bc)) in enumerate(zip(lat, shapes)):
        dom = dict(nx=s[0], ny=s[1], nz=s[2], nu=0.01 + 0.005 * i, bc=bc, body_force=(1e-5, 0.0, 2e-6))
        ref, _ = _run_aa(dom, "bf16", (32, 4), 2, (6,), state=states[i])
        np.testing.assert_array_equal(L.pdfs(), ref[-1])
    for L in lat:
        L.destroy()


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
def test_paired_bulk_beside_a_rotor_at_a_wall_face(coll):
    """A rotor whose force box comes within a tile of a free-slip face: rotor
    tiles on the face, face tiles (one cell per thread) and the paired bulk in
    one step, bit for bit the one-cell form's results."""
    dom, turb = I.single_turbine_case(64, 34, 40, diameter=16.0, elements_per_blade=8, seed=779)
    dom["collision"] = coll
    dom["bc"] = ("inout", "freeslip", "periodic")
    a = _run(dom, "bf16", (32, 4), 0, 12, turb=turb, inflow=True, diag_every=5)
    b = _run(dom, "bf16", (32, 4), 2, 12, turb=turb, inflow=True, diag_every=5)
    _same(a, b)


def test_tiles_of_partial_warps_keep_one_cell():
    """Tiles of 32 x 1 and 32 x 3 cells would give paired CTAs of 16 and 48
    threads, not whole warps: the two-array and in-place steps then run one cell
    per thread, with diagnostics, and agree with the one-cell form."""
    dom = dict(nx=64, ny=9, nz=4, nu=0.02, body_force=(2e-6, 0.0, 0.0))
    state = I.random_state(64, 9, 4, seed=5)
    for tile in ((32, 1), (32, 3)):
        a = _run(dom, "bf16", tile, 0, 5, state=state, diag_every=2)
        b = _run(dom, "bf16", tile, 2, 5, state=state, diag_every=2)
        np.testing.assert_array_equal(a["pdfs"], b["pdfs"])
        np.testing.assert_array_equal(a["diag"][0], b["diag"][0])
        assert a["diag"][1] == b["diag"][1]
        c, _ = _run_aa(dom, "bf16", tile, 0, (2, 2), state=state, diag_every=2)
        d, _ = _run_aa(dom, "bf16", tile, 2, (2, 2), state=state, diag_every=2)
        for u, v in zip(c, d):
            np.testing.assert_array_equal(u, v)
