"""Pins of the oracle's time stepping against closed-form flows.

Decaying shear wave and z-invariant Taylor-Green vortex are exact
Navier-Stokes solutions; the 3-D Taylor-Green vortex at small amplitude
follows its Stokes-limit decay; body-force Poiseuille flow between halfway
bounce-back walls has a parabolic closed form, and with a Smagorinsky eddy
viscosity its gradient solves (nu + C^2 |g|) g = -F (y - y_c) pointwise.
Tolerances come from the observed second-order convergence where stated.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2402_13171_gb300 import inputs as I

C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], dtype=np.float64)


def kinetic_energy(sim):
    rho, u = sim.moments()
    return 0.5 * np.sum(rho * (u ** 2).sum(0))


def shear_wave_nu(ny, nu, steps, coll="cumulant"):
    d = O.make_domain(1, ny, 1, collision=coll, nu=nu)
    s = O.Sim(d)
    rho, u = I.shear_wave(1, ny, 1, 1e-3)
    s.init_fields(rho, u)
    k = 2 * math.pi / ny
    prof = np.sin(k * np.arange(ny))
    amps = []
    for n in (20, steps):
        s.step(n - s.step_count)
        amps.append(np.dot(s.moments()[1][0, 0, :, 0], prof) / np.dot(prof, prof))
    return -math.log(amps[1] / amps[0]) / (k * k * (steps - 20))


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
def test_shear_wave_viscosity_converges(coll):
    nu = 0.05
    e16 = abs(shear_wave_nu(16, nu, 220, coll) / nu - 1)
    e32 = abs(shear_wave_nu(32, nu, 420, coll) / nu - 1)
    assert e32 < 5e-3
    assert e16 / e32 > 3.0   # second order in k


def tgv_nu_ratio(n, u0, nu, steps, three_d=False):
    """Viscosity seen by the Taylor-Green energy decay between steps/10 and
    steps (after the start-up transient of an equilibrium initial state)."""
    d = O.make_domain(n, n, n if three_d else 1, nu=nu)
    s = O.Sim(d)
    rho, u = I.taylor_green_3d(n, u0) if three_d else I.taylor_green_2d(n, u0)
    s.init_fields(rho, u)
    s.step(steps // 10)
    E1 = kinetic_energy(s)
    s.step(steps - steps // 10)
    E2 = kinetic_energy(s)
    k = 2 * math.pi / n
    return -math.log(E2 / E1) / (steps - steps // 10) / ((6 if three_d else 4) * k * k) / nu


def test_taylor_green_2d_exact_decay():
    """z-invariant vortex: E ~ exp(-4 nu k^2 t) exactly; the lattice error
    shrinks under diffusive scaling (u0 ~ 1/n, steps ~ n^2)."""
    e32 = abs(tgv_nu_ratio(32, 0.05, 0.01, 200) - 1)
    e64 = abs(tgv_nu_ratio(64, 0.025, 0.01, 800) - 1)
    assert e32 < 1.5e-2
    assert e64 < 0.5 * e32


def test_taylor_green_3d_stokes_limit():
    """3-D vortex at small amplitude: E ~ exp(-6 nu k^2 t); the lattice error
    falls at second order from 16^3 to 24^3."""
    e16 = abs(tgv_nu_ratio(16, 0.005, 0.01, 100, three_d=True) - 1)
    e24 = abs(tgv_nu_ratio(24, 0.005, 0.01, 200, three_d=True) - 1)
    assert e24 < 1.5e-2
    assert e16 / e24 > 2.0


def poiseuille_error(ny, coll, nu=0.1, F=1e-6):
    d = O.make_domain(1, ny, 1, collision=coll, nu=nu, bc=("periodic", "noslip", "periodic"), body_force=(F, 0, 0))
    s = O.Sim(d)
    s.init_fields()
    t_diff = ny * ny / (math.pi ** 2 * nu)
    s.step(int(14 * t_diff))
    ux = s.moments()[1][0, 0, :, 0]
    y = np.arange(ny)
    exact = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    return np.abs(ux - exact).max() / exact.max()


@pytest.mark.parametrize("coll", ["cumulant", "srt_smag"])
def test_body_force_poiseuille(coll):
    e8 = poiseuille_error(8, coll)
    e16 = poiseuille_error(16, coll)
    assert e16 < 2e-2
    assert e8 / e16 > 3.0 or e16 < 1e-6


def test_smagorinsky_poiseuille_closed_form():
    ny, nu, Cs, F = 16, 0.05, 1.0, 1e-4
    d = O.make_domain(1, ny, 1, collision="srt_smag", nu=nu, smag_c=Cs, bc=("periodic", "noslip", "periodic"),
                      body_force=(F, 0, 0))
    s = O.Sim(d)
    s.init_fields()
    s.step(6000)
    ux = s.moments()[1][0, 0, :, 0]
    y = np.arange(ny)
    yc = (ny - 1) / 2.0
    g_meas = (ux[2:] - ux[:-2]) / 2.0
    src = -F * (y[1:-1] - yc)
    g = np.sign(src) * (-nu + np.sqrt(nu * nu + 4 * Cs * Cs * np.abs(src))) / (2 * Cs * Cs)
    inner = slice(1, -1)
    assert np.abs(g_meas[inner] - g[inner]).max() < 0.03 * np.abs(g).max()
    # the eddy viscosity is a sizeable part: a laminar fit would miss by far more
    g_lam = src / nu
    assert np.abs(g_meas[inner] - g_lam[inner]).max() > 0.15 * np.abs(g).max()


# ------------------------------------------------------------- streaming rules

def test_pull_periodic_is_a_shift():
    rng = np.random.default_rng(11)
    nx, ny, nz = 5, 4, 3
    d = O.make_domain(nx, ny, nz)
    s = O.Sim(d)
    f = rng.uniform(0, 1, (27, nz, ny, nx))
    for (x, y, z) in [(0, 0, 0), (4, 3, 2), (2, 1, 1)]:
        out = s.pull_cell(f, 0, x, y, z)
        for q in range(27):
            cx, cy, cz = C[q].astype(int)
            assert out[q] == f[q, (z - cz) % nz, (y - cy) % ny, (x - cx) % nx]


def test_pull_bounce_back_inlet_outlet():
    rng = np.random.default_rng(12)
    nx, ny, nz = 6, 5, 4
    d = O.make_domain(nx, ny, nz, bc=("inout", "noslip", "periodic"), u_ref=(0.05, 0, 0), noise_rel=0.0)
    s = O.Sim(d)
    f = rng.uniform(0, 1, (27, nz, ny, nx))
    feq_in = O.equilibrium(1.0, [0.05, 0, 0])
    for (x, y, z) in [(0, 0, 1), (nx - 1, ny - 1, 3), (0, 2, 0), (nx - 1, 2, 2), (3, 0, 2)]:
        out = s.pull_cell(f, 0, x, y, z)
        for q in range(27):
            cx, cy, cz = C[q].astype(int)
            sx, sy, sz = x - cx, y - cy, (z - cz) % nz
            if sy < 0 or sy >= ny:
                assert out[q] == f[26 - q, z, y, x]
            elif sx < 0:
                assert out[q] == feq_in[q]
            elif sx >= nx:
                assert out[q] == f[q, sz, sy, nx - 1]
            else:
                assert out[q] == f[q, sz, sy, sx]


def test_uniform_inflow_state_is_steady():
    d = O.make_domain(12, 6, 5, bc=("inout", "periodic", "periodic"), u_ref=(0.05, 0.01, 0), noise_rel=0.0, nu=0.01)
    s = O.Sim(d)
    s.init_fields()
    f0 = s.f.copy()
    s.step(5)
    np.testing.assert_allclose(s.f, f0, atol=2e-16)


def _inflow(d, step, y, z):
    return O.inflow_velocity(d, step, y, z)


def test_log_law_inflow_profile():
    """The farm's log-law inflow (a reading of the configuration): the mean
    profile is zero at the roughness height z_c = z0, equals u_ref at z_c =
    z_ref, and is logarithmic, rising by the same amount over every equal
    ratio of heights (here 1/2, 3/2, 9/2, 27/2 at ratio 3, each step
    u_ref ln 3 / ln(z_ref / z0)); at the three cell centres z_c = 2.5, 6.5 and
    11.5 it is u_ref ln(z_c/z0)/ln(z_ref/z0)."""
    u_ref, z0, z_ref = 0.05, 0.5, 13.5
    d = O.make_domain(4, 3, 16, bc=("inout", "periodic", "freeslip"), inflow_kind=1, u_ref=(u_ref, 0, 0), z0=z0,
                      z_ref=z_ref, noise_rel=0.0)
    u = np.array([_inflow(d, 0, 1, z) for z in range(16)])
    assert u[0, 0] == 0.0                                   # z_c = 0.5 = z0
    assert u[13, 0] == pytest.approx(u_ref, rel=1e-15)     # z_c = 13.5 = z_ref
    inc = u_ref * math.log(3.0) / math.log(z_ref / z0)
    for z_lo, z_hi in ((0, 1), (1, 4), (4, 13)):            # z_c ratio 3
        assert u[z_hi, 0] - u[z_lo, 0] == pytest.approx(inc, rel=1e-13)
    for z in (2, 6, 11):
        zc = z + 0.5
        assert u[z, 0] == pytest.approx(u_ref * math.log(zc / z0) / math.log(z_ref / z0), rel=1e-14)
    np.testing.assert_array_equal(u[:, 1:], 0.0)
    assert np.all(np.diff(u[:, 0]) > 0)


def test_log_law_inflow_shares_the_noise_of_the_uniform_inflow():
    """The seeded noise does not depend on the mean profile: at every step,
    column and component the log-law inflow minus the uniform one is exactly
    the difference of the means, and the noise amplitude is noise_rel |u_ref|
    at every height."""
    kw = dict(bc=("inout", "periodic", "freeslip"), u_ref=(0.04, 0.01, 0.0), noise_rel=0.01, seed=99)
    d_log = O.make_domain(4, 5, 12, inflow_kind=1, z0=0.1, z_ref=6.0, **kw)
    d_uni = O.make_domain(4, 5, 12, inflow_kind=0, **kw)
    amp = 0.01 * math.hypot(0.04, 0.01)
    for step in (0, 3, 1000):
        for y, z in ((0, 0), (2, 5), (4, 11)):
            scale = math.log((z + 0.5) / 0.1) / math.log(6.0 / 0.1)
            ul, uu = _inflow(d_log, step, y, z), _inflow(d_uni, step, y, z)
            np.testing.assert_allclose(ul - uu, np.array([0.04, 0.01, 0.0]) * (scale - 1.0), rtol=0, atol=1e-17)
            assert np.all(np.abs(uu - np.array([0.04, 0.01, 0.0])) <= amp)


def test_log_law_initial_state_is_the_mean_profile():
    """With no velocity given the oracle starts from the equilibrium of the
    mean inflow, the log profile on a log-law lattice."""
    d = O.make_domain(5, 3, 10, bc=("inout", "periodic", "freeslip"), inflow_kind=1, u_ref=(0.05, 0, 0), z0=0.1,
                      z_ref=5.0, noise_rel=0.0)
    s = O.Sim(d)
    s.init_fields()
    rho, u = s.moments()
    prof = I.log_law_profile(10, 0.05, 0.1, 5.0)
    np.testing.assert_allclose(rho, 1.0, atol=1e-15)
    np.testing.assert_allclose(u[0], np.broadcast_to(prof[:, None, None], u[0].shape), atol=1e-16)
    np.testing.assert_allclose(u[1:], 0.0, atol=1e-16)


def test_mass_and_momentum_conserved_periodic():
    rng_state = I.random_state(6, 5, 7, seed=99, u_mean=(0.02, -0.01, 0.01))
    for coll in ("cumulant", "srt_smag"):
        d = O.make_domain(6, 5, 7, collision=coll, nu=0.02, smag_c=0.1, body_force=(1e-5, 2e-5, -1e-5))
        s = O.Sim(d)
        s.init_fields(*rng_state)
        m0 = s.f.sum()
        j0 = np.einsum("qa,qzyx->a", C, s.f)
        s.step(3)
        assert s.f.sum() == pytest.approx(m0, rel=1e-14)
        np.testing.assert_allclose(np.einsum("qa,qzyx->a", C, s.f), j0 + 3 * 6 * 5 * 7 * np.array([1e-5, 2e-5, -1e-5]),
                                   atol=1e-13)


def test_pull_free_slip_reflects():
    rng = np.random.default_rng(13)
    nx, ny, nz = 5, 4, 6
    d = O.make_domain(nx, ny, nz, bc=("periodic", "periodic", "freeslip"))
    s = O.Sim(d)
    f = rng.uniform(0, 1, (27, nz, ny, nx))
    for (x, y, z) in [(0, 0, 0), (2, 3, nz - 1), (4, 1, 3)]:
        out = s.pull_cell(f, 0, x, y, z)
        for q in range(27):
            cx, cy, cz = C[q].astype(int)
            sz = z - cz
            if sz < 0 or sz >= nz:
                qm = (-cz + 1) * 9 + (cy + 1) * 3 + (cx + 1)
                assert out[q] == f[qm, z, (y - cy) % ny, (x - cx) % nx]
            else:
                assert out[q] == f[q, sz, (y - cy) % ny, (x - cx) % nx]


def test_free_slip_channel_uniform_flow_is_steady():
    d = O.make_domain(6, 5, 8, bc=("periodic", "periodic", "freeslip"), u_ref=(0.05, 0.02, 0.0), nu=0.02)
    s = O.Sim(d)
    s.init_fields()
    f0 = s.f.copy()
    s.step(4)
    np.testing.assert_allclose(s.f, f0, atol=2e-16)


def free_slip_wave_nu(nz, nu, steps):
    """u_x = u0 cos(pi (z + 1/2) / nz) between free-slip walls at z = -1/2 and
    nz - 1/2 (zero shear stress) decays as exp(-nu k^2 t), k = pi / nz."""
    d = O.make_domain(1, 1, nz, nu=nu, bc=("periodic", "periodic", "freeslip"))
    s = O.Sim(d)
    k = math.pi / nz
    z = np.arange(nz) + 0.5
    u = np.zeros((3, nz, 1, 1))
    u[0, :, 0, 0] = 1e-3 * np.cos(k * z)
    s.init_fields(np.ones(nz), u)
    prof = np.cos(k * z)
    amps = []
    for n in (20, steps):
        s.step(n - s.step_count)
        amps.append(np.dot(s.moments()[1][0, :, 0, 0], prof) / np.dot(prof, prof))
    return -math.log(amps[1] / amps[0]) / (k * k * (steps - 20))


def test_free_slip_wave_decay_converges():
    nu = 0.05
    e8 = abs(free_slip_wave_nu(8, nu, 120) / nu - 1)
    e16 = abs(free_slip_wave_nu(16, nu, 420) / nu - 1)
    assert e16 < 2e-2
    assert e8 / e16 > 3.0
