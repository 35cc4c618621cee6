"""The batched sweep at full size (16 seeded single-rotor lattices, 71.9 M
cells) in the launch configurations the benchmark's tuner picks (32x4x1 with
rotor tiles of 3 planes; 32x4x8, z-marching): one batched step from seeded
near-equilibrium states, checked against the FP64 oracle lattice by lattice on
every element force and rotor load and on sampled cells (next to blade
elements, inlet, outlet, bulk).

Tolerances as in the single-lattice full-size test: element positions 2e-5,
element forces 1e-5 of the largest, loads 1e-5 relative, PDFs 2e-7 absolute.
"""
import numpy as np
import pytest

import oracle as O
from paper_2402_13171_gb300 import inputs as I
from cases import oracle_sim

pytestmark = pytest.mark.gpu

F_TOL = 2e-7


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_13171_gb300 import build
    build.build()
    O.build()


def _state(i, dom):
    return I.random_state(dom["nx"], dom["ny"], dom["nz"], seed=7000 + i, u_mean=(dom["u_ref"][0], 0.0, 0.0),
                          du=0.005, drho=0.002, fneq_amp=2e-4)


@pytest.mark.parametrize("tile", [(32, 4, 1), (32, 4, 8)])
def test_full_size_batch16_sampled(tile):
    from paper_2402_13171_gb300 import lbm
    cases = I.batch_instances(16)
    cfgs = [dict(nx=d["nx"], ny=d["ny"], nz=d["nz"], collision=d["collision"], nu=d["nu"], smag_c=d["smag_c"],
                 bc=d["bc"], seed=d["seed"], tile=tile) for d, _ in cases]
    lat = lbm.batch_create(cfgs)
    assert sum(L.N for L in lat) == 71866368
    before = []
    for i, (L, (d, t)) in enumerate(zip(lat, cases)):
        L.set_inflow(u_ref=d["u_ref"], noise_rel=d["noise_rel"])
        L.add_turbine(**t)
        rho, u, fneq = _state(i, d)
        L.init_fields(rho, u, fneq)
        before.append(L.loads(0, elements=True))
    assert lat[0].tile()[:3] == tile
    lat[0].step(1)
    rng = np.random.default_rng(77)
    for i, (L, (d, t)) in enumerate(zip(lat, cases)):
        nx, ny, nz = d["nx"], d["ny"], d["nz"]
        s = oracle_sim(d, [t])
        rho, u, fneq = _state(i, d)
        s.init_fields(rho, u, fneq)
        del rho, u, fneq
        f0 = s.f
        pos, fb, alpha, loads = s.alm_forces(f0, np.zeros((3, nz, ny, nx)), 0)
        th, tq, ef, ep = before[i]
        np.testing.assert_allclose(ep, pos, atol=2e-5, err_msg=f"lattice {i}")
        np.testing.assert_allclose(ef, fb, atol=1e-5 * np.abs(fb).max(), err_msg=f"lattice {i}")
        assert th == pytest.approx(loads[0], rel=1e-5), i
        assert tq == pytest.approx(loads[1], rel=1e-5), i
        fg = L.pdfs()
        hub = np.round(np.array(t["hub"])).astype(int)
        cells = [(0, 0, 0), (0, ny // 2, nz // 3), (nx - 1, ny - 1, nz - 1), (nx - 1, 3, nz // 2), tuple(hub)]
        cells += [tuple(int(v) for v in np.round(p)) for p in pos[::12]]
        cells += [tuple(int(v) for v in c) for c in rng.integers([0, 0, 0], [nx, ny, nz], (4, 3))]
        for (x, y, z) in cells:
            F = O.spread_at(pos, fb, t["epsilon"], x, y, z, kernel=t["kernel"])
            ref = s.update_cell(f0, F, 0, x, y, z)
            np.testing.assert_allclose(fg[:, z, y, x], ref, atol=F_TOL, rtol=0, err_msg=f"lattice {i} {(x, y, z)}")
        del fg, s, f0
