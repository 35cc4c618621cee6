"""Pins of the oracle's actuator line against geometry and blade-element theory.

Kinematics against the circle the blades trace; element forces in a frozen
uniform field against the textbook blade-element split into thrust
(C_L cos phi + C_D sin phi) and driving force (C_L sin phi - C_D cos phi);
trilinear sampling against hat-function interpolation of brute-force pulled
moments; Gaussian spreading against the force-sum identity and the continuous
Gaussian's unit mass; the Roma delta against the three moment conditions it is
built from; polar lookup against its nodes.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2402_13171_gb300 import inputs as I

C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], dtype=np.float64)


def make_turbine(**kw):
    t = I.single_turbine(64, 48, 48, diameter=16.0, hub=(20.0, 24.0, 24.0), elements_per_blade=8, **kw)
    return O.TurbineSpec(**t), t


def test_kinematics_circle():
    T, t = make_turbine()
    R, ne = t["radius"], t["n_elements"]
    hub = np.array(t["hub"])
    for step in (0, 7, 123):
        for b in range(3):
            for k in (0, 3, 7):
                e = O.element_kinematics(T, step, b, k)
                r = (k + 0.5) * R / ne
                assert e["r"] == pytest.approx(r)
                rel = e["pos"] - hub
                assert np.linalg.norm(rel) == pytest.approx(r, rel=1e-14)
                assert rel[0] == pytest.approx(0.0, abs=1e-14)  # rotor plane x = hub_x (no yaw)
                theta = t["omega"] * step + 2 * math.pi * b / 3
                np.testing.assert_allclose(rel, r * np.array([0, math.cos(theta), math.sin(theta)]), atol=1e-13)
                # rigid rotation about +x
                np.testing.assert_allclose(e["vel"], t["omega"] * np.cross([1, 0, 0], rel), atol=1e-15)
                np.testing.assert_allclose(e["e_t"], np.cross(e["e_axis"], e["e_r"]), atol=1e-15)


def test_kinematics_yaw_turns_axis():
    T, t = make_turbine(yaw=math.radians(90))
    e = O.element_kinematics(T, 0, 0, 0)
    np.testing.assert_allclose(e["e_axis"], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(e["e_r"], [-1, 0, 0], atol=1e-15)


def uniform_sim(U, nx=64, ny=48, nz=48, **tk):
    d = O.make_domain(nx, ny, nz, bc=("periodic",) * 3, u_ref=(U, 0, 0))
    T, t = make_turbine(**tk)
    s = O.Sim(d, [T])
    s.init_fields()
    return s, T, t


def test_frozen_field_blade_element_forces():
    U = 0.05
    s, T, t = uniform_sim(U)
    pos, fb, alpha, loads = s.alm_forces(s.f, s.falm, 0)
    R, ne, Om = t["radius"], t["n_elements"], t["omega"]
    l = R / ne
    thrust = torque = 0.0
    for k in range(ne):
        r = (k + 0.5) * l
        W = math.hypot(U, Om * r)
        phi = math.atan2(U, Om * r)
        CL = np.interp(phi, t["alpha"], t["cl"])
        CD = np.interp(phi, t["alpha"], t["cd"])
        c = t["chord_root"] + (t["chord_tip"] - t["chord_root"]) * r / R
        q = 0.5 * W * W * c * l
        f_axial = q * (CL * math.cos(phi) + CD * math.sin(phi))
        f_tang = q * (CL * math.sin(phi) - CD * math.cos(phi))
        assert alpha[k] == pytest.approx(phi, abs=1e-12)
        # blade 0 at theta = 0: e_r = +y, e_t = +z
        np.testing.assert_allclose(fb[k], [f_axial, 0.0, f_tang], rtol=1e-10, atol=1e-16)
        thrust += 3 * f_axial
        torque += 3 * r * f_tang
    assert loads[0] == pytest.approx(thrust, rel=1e-10)
    assert loads[1] == pytest.approx(torque, rel=1e-10)
    assert loads[0] > 0 and loads[1] > 0   # thrust downstream, driving torque


def test_tip_loss_factor_values_and_limits():
    """Glauert's tip-loss factor in Prandtl's form, F = (2/pi) arccos(e^-f),
    f = B (R - r) / (2 r |sin phi|): F = 2/3 where f = ln 2 (arccos 1/2 =
    pi/3), F = 1/2 where e^-f = cos(pi/4); F = 0 at the tip, F -> 1 far
    inboard or for sin phi -> 0, even in phi, rising with the blade count."""
    B, R = 3, 16.0
    # choose r so that f = ln 2 at phi = 0.3
    phi = 0.3
    r = B * R / (B + 2 * math.log(2) * math.sin(phi))
    assert O.tip_loss(B, R, r, phi) == pytest.approx(2.0 / 3.0, abs=1e-14)
    f = -math.log(math.cos(math.pi / 4))
    r = B * R / (B + 2 * f * math.sin(phi))
    assert O.tip_loss(B, R, r, phi) == pytest.approx(0.5, abs=1e-14)
    assert O.tip_loss(B, R, R, phi) == 0.0
    assert O.tip_loss(B, R, 0.5, phi) == pytest.approx(1.0, abs=1e-12)
    assert O.tip_loss(B, R, 15.0, 0.0) == 1.0
    assert O.tip_loss(B, R, 15.0, 1e-9) == pytest.approx(1.0, abs=1e-12)
    for rr in (4.0, 12.0, 15.5):
        assert O.tip_loss(B, R, rr, -phi) == O.tip_loss(B, R, rr, phi)
        assert O.tip_loss(2, R, rr, phi) < O.tip_loss(3, R, rr, phi) < O.tip_loss(6, R, rr, phi)
    Fs = [O.tip_loss(B, R, rr, phi) for rr in np.linspace(1.0, R, 40)]
    assert all(a >= b for a, b in zip(Fs, Fs[1:]))


def test_frozen_field_tip_loss_scales_each_element():
    """In a frozen uniform field the tip-loss option multiplies each element
    force by its factor at the element's inflow angle and nothing else, and it
    takes thrust and torque down."""
    U = 0.05
    s0, _, t = uniform_sim(U)
    s1, _, _ = uniform_sim(U, tip_loss=True)
    pos0, fb0, alpha0, loads0 = s0.alm_forces(s0.f, s0.falm, 0)
    pos1, fb1, alpha1, loads1 = s1.alm_forces(s1.f, s1.falm, 0)
    np.testing.assert_array_equal(alpha0, alpha1)
    R, ne = t["radius"], t["n_elements"]
    for e in range(fb0.shape[0]):
        r = (e % ne + 0.5) * R / ne
        F = O.tip_loss(3, R, r, alpha0[e])
        np.testing.assert_allclose(fb1[e], F * fb0[e], rtol=1e-13, atol=1e-18)
    assert fb1[ne - 1, 0] < 0.7 * fb0[ne - 1, 0]      # outermost element loses most
    assert fb1[0, 0] > 0.99 * fb0[0, 0]               # innermost hardly at all
    assert 0 < loads1[0] < loads0[0] and 0 < loads1[1] < loads0[1]


def test_sampling_is_hat_interpolation_of_pulled_moments():
    rng = np.random.default_rng(21)
    nx, ny, nz = 8, 7, 6
    d = O.make_domain(nx, ny, nz, body_force=(1e-4, 0, -2e-4))
    s = O.Sim(d)
    rho, u, fneq = I.random_state(nx, ny, nz, seed=5)
    s.init_fields(rho, u, fneq)
    falm = rng.uniform(-1e-3, 1e-3, (3, nz, ny, nx))
    f = s.f
    # brute force: pulled populations by periodic rolls, then moments per cell
    pulled = np.stack([np.roll(f[q], shift=(int(C[q, 2]), int(C[q, 1]), int(C[q, 0])), axis=(0, 1, 2))
                       for q in range(27)])
    R = pulled.sum(0)
    Ftot = falm + np.array([1e-4, 0, -2e-4])[:, None, None, None]
    Uc = (np.einsum("qa,qzyx->azyx", C, pulled) + 0.5 * Ftot) / R
    for p in ([3.3, 2.7, 4.1], [0.0, 6.5, 5.9], [7.25, 0.5, 0.0]):
        wsum = 0.0
        r_ref = 0.0
        u_ref = np.zeros(3)
        for z in range(nz + 1):
            for y in range(ny + 1):
                for x in range(nx + 1):
                    w = max(0, 1 - abs(x - p[0])) * max(0, 1 - abs(y - p[1])) * max(0, 1 - abs(z - p[2]))
                    if w == 0:
                        continue
                    wsum += w
                    r_ref += w * R[z % nz, y % ny, x % nx]
                    u_ref += w * Uc[:, z % nz, y % ny, x % nx]
        assert wsum == pytest.approx(1.0)
        r, uu = s.sample(f, falm, 0, p)
        assert r == pytest.approx(r_ref, abs=1e-14)
        np.testing.assert_allclose(uu, u_ref, atol=1e-15)


def test_gaussian_axis_mass():
    """By Poisson summation the untruncated lattice sum of the 1-D Gaussian
    exp(-s^2/eps^2)/(eps sqrt(pi)) is 1 up to ~exp(-pi^2 eps^2); the sum cut at
    3 eps is therefore 1 minus the discrete tail beyond 3 eps."""
    for eps in (1.5, 2.0, 3.0):
        for p in (0.0, 0.3, 17.77):
            i = np.arange(math.floor(p) - 60, math.floor(p) + 61)
            s = i - p
            tail = np.sum(np.exp(-s[np.abs(s) > 3 * eps] ** 2 / eps ** 2)) / (eps * math.sqrt(math.pi))
            assert O.gauss_axis_sum(p, eps) == pytest.approx(1.0 - tail, abs=2.5 * math.exp(-math.pi ** 2 * eps ** 2) + 1e-14)
            assert 1e-6 < tail < 1e-4


def test_spread_force_sum_and_support():
    d = O.make_domain(40, 40, 40)
    rng = np.random.default_rng(22)
    pos = rng.uniform(12, 28, (5, 3))
    fb = rng.uniform(-1, 1, (5, 3))
    eps = 2.0
    force = O.spread(d, pos, fb, eps)
    np.testing.assert_allclose(force.reshape(3, -1).sum(1), -fb.sum(0), atol=1e-13)
    # single element: zero beyond 3 eps per axis, separable and centred
    f1 = O.spread(d, pos[:1], fb[:1], eps)
    nz_idx = np.argwhere(np.abs(f1[0]) > 0)
    p = pos[0]
    assert np.all(np.abs(nz_idx[:, ::-1] - p) <= 3 * eps + 1e-12)
    x0, y0, z0 = np.round(p).astype(int)
    w = f1[0] / -fb[0, 0]
    gx = np.exp(-((np.arange(40) - p[0]) ** 2) / eps ** 2)
    # ratio of weights along x at fixed (y0, z0) follows the 1-D Gaussian
    assert w[z0, y0, x0 + 1] / w[z0, y0, x0] == pytest.approx(gx[x0 + 1] / gx[x0], rel=1e-12)
    # spread_at agrees with the scatter
    for (x, y, z) in [(x0, y0, z0), (x0 + 2, y0 - 3, z0 + 1)]:
        np.testing.assert_allclose(O.spread_at(pos, fb, eps, x, y, z), force[:, z, y, x], atol=1e-15)


def _roma_samples(r):
    """phi(r - j) at every integer j with a non-zero sample."""
    j = np.arange(math.floor(r) - 3, math.floor(r) + 4)
    return j, np.array([O.roma_phi(r - jj) for jj in j])


def test_roma_delta_moment_conditions():
    """Roma, Peskin and Berger (1999) construct their three-point delta from
    three conditions on its integer-shifted samples, for every shift r: they
    sum to 1, their first moment about r vanishes, and their squares sum to
    1/2.  A wrong constant, sign or branch breaks at least one of them."""
    rng = np.random.default_rng(31)
    for r in np.concatenate([np.linspace(-2.0, 2.0, 81), rng.uniform(-40, 40, 200)]):
        j, ph = _roma_samples(r)
        assert np.all(ph >= 0)
        assert ph.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.dot(r - j, ph) == pytest.approx(0.0, abs=1e-14)
        assert np.dot(ph, ph) == pytest.approx(0.5, abs=1e-14)
        assert np.count_nonzero(ph) <= 3


def test_roma_delta_values_and_continuity():
    assert O.roma_phi(0.0) == pytest.approx(2.0 / 3.0, abs=1e-16)
    for r in (0.5, -0.5):
        assert O.roma_phi(r) == pytest.approx(0.5, abs=1e-15)
    for r in (1.5, -1.5, 1.7, -3.0):
        assert O.roma_phi(r) == 0.0
    for r0 in (0.5, 1.5):
        for dr in (1e-9, 1e-11):
            assert O.roma_phi(r0 - dr) == pytest.approx(O.roma_phi(r0 + dr), abs=1e-4)
    for r in np.linspace(0, 1.6, 17):
        assert O.roma_phi(r) == O.roma_phi(-r)


def test_roma_spread_force_sum_centroid_and_support():
    """With the Roma delta every element's spread force sums to the element
    force and its force-weighted centroid is the element position (the first
    moment condition, per axis), with support |x_a - p_a| < 3/2."""
    d = O.make_domain(24, 24, 24)
    rng = np.random.default_rng(23)
    pos = rng.uniform(6, 18, (5, 3))
    fb = rng.uniform(-1, 1, (5, 3))
    force = O.spread(d, pos, fb, 2.0, kernel="roma")
    np.testing.assert_allclose(force.reshape(3, -1).sum(1), -fb.sum(0), atol=1e-14)
    f1 = O.spread(d, pos[:1], fb[:1], 2.0, kernel="roma")
    w = f1[0] / -fb[0, 0]
    assert w.sum() == pytest.approx(1.0, abs=1e-14)
    zz, yy, xx = np.meshgrid(np.arange(24), np.arange(24), np.arange(24), indexing="ij")
    for a, g in enumerate((xx, yy, zz)):
        assert (w * g).sum() == pytest.approx(pos[0, a], abs=1e-12)
    nz_idx = np.argwhere(w != 0)
    assert np.all(np.abs(nz_idx[:, ::-1] - pos[0]) < 1.5)
    assert len(nz_idx) <= 27
    # epsilon plays no part
    np.testing.assert_array_equal(O.spread(d, pos, fb, 4.0, kernel="roma"), force)
    x0, y0, z0 = np.round(pos[0]).astype(int)
    for (x, y, z) in [(x0, y0, z0), (x0 + 1, y0 - 1, z0), (x0 + 2, y0, z0)]:
        np.testing.assert_allclose(O.spread_at(pos, fb, 2.0, x, y, z, kernel="roma"), force[:, z, y, x],
                                   atol=1e-15)


def test_polar_lookup():
    a, cl, cd = I.synthetic_polars()
    assert O.table_lookup(a, cl, a[1000]) == cl[1000]
    mid = 0.5 * (a[1800] + a[1801])
    assert O.table_lookup(a, cl, mid) == pytest.approx(0.5 * (cl[1800] + cl[1801]))
    assert O.table_lookup(a, cd, 10.0) == cd[-1]
    assert O.table_lookup(a, cd, -10.0) == cd[0]
    # within table spacing of the analytic polar on the linear part
    x = math.radians(5.03)
    assert O.table_lookup(a, cl, x) == pytest.approx(2 * math.pi * x, abs=1e-12)
    assert O.table_lookup(a, cd, x) == pytest.approx(0.01 + 0.02 * x * x, abs=0.02 * math.radians(0.1) ** 2)


@pytest.mark.parametrize("kernel", ["gauss", "roma"])
def test_alm_step_momentum_balance(kernel):
    """Over one step the fluid momentum changes by exactly minus the sum of the
    blade forces (the spread conserves force)."""
    s, T, t = uniform_sim(0.05, kernel=kernel)
    j0 = np.einsum("qa,qzyx->a", C, s.f)
    s.step(1)
    j1 = np.einsum("qa,qzyx->a", C, s.f)
    # rounding of a sum of ~1.5e5 cells with total momentum ~7e3
    np.testing.assert_allclose(j1 - j0, -s.elem_force.sum(0), atol=1e-10)
    assert s.loads[0, 0] > 0


# ------------------------------------------------ yaw, twist, pitch, unequal polar tables

def _frame(yaw, theta):
    """Rotor frame of a blade at azimuth theta on a rotor yawed by `yaw` about
    +z, built from its geometric definition: the axis is the horizontal unit
    vector at angle yaw from +x, blade 0 at theta = 0 is horizontal and points
    to the left of the axis, and theta turns it positively about the axis (up
    through +z at theta = pi/2)."""
    ea = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    left = np.array([-math.sin(yaw), math.cos(yaw), 0.0])
    up = np.array([0.0, 0.0, 1.0])
    er = math.cos(theta) * left + math.sin(theta) * up
    return ea, er, np.cross(ea, er)


def test_kinematics_yaw_at_closed_form_points():
    """A yawed rotor (7 degrees) with a start angle: every element lies in the
    plane through the hub normal to the tilted axis, at its radius, on the
    blade direction of its azimuth; the rigid rotation gives its velocity."""
    yaw, theta0 = math.radians(7.0), 0.3
    t = I.single_turbine(64, 48, 48, diameter=16.0, hub=(20.0, 24.0, 24.0), elements_per_blade=8, yaw=yaw)
    t["theta0"] = theta0
    T = O.TurbineSpec(**t)
    hub = np.array(t["hub"])
    for step in (0, 11, 400):
        for b in range(3):
            theta = theta0 + t["omega"] * step + 2 * math.pi * b / 3
            ea, er, et = _frame(yaw, theta)
            for k in (0, 5, 7):
                e = O.element_kinematics(T, step, b, k)
                r = (k + 0.5) * t["radius"] / t["n_elements"]
                np.testing.assert_allclose(e["e_axis"], ea, atol=1e-15)
                np.testing.assert_allclose(e["e_r"], er, atol=1e-13)
                np.testing.assert_allclose(e["e_t"], et, atol=1e-13)
                np.testing.assert_allclose(e["pos"], hub + r * er, atol=1e-12)
                assert np.dot(e["pos"] - hub, ea) == pytest.approx(0.0, abs=1e-13)
                np.testing.assert_allclose(e["vel"], t["omega"] * r * et, atol=1e-15)


def _skewed_element(U, yaw, Om, r, theta):
    """Blade-element inflow of a yawed rotor in a uniform stream U e_x: the
    stream has axial part U cos(yaw), radial part -U sin(yaw) cos(theta)
    (removed), and tangential part U sin(yaw) sin(theta), against the blade's
    own speed Om r; returns (phi, |u_rel|^2)."""
    ua = U * math.cos(yaw)
    ut = U * math.sin(yaw) * math.sin(theta) - Om * r
    return math.atan2(ua, -ut), ua * ua + ut * ut


@pytest.mark.parametrize("yaw_deg,twisted", [(7.0, False), (7.0, True), (25.0, True)])
def test_frozen_field_yawed_twisted_pitched_forces(yaw_deg, twisted):
    """Frozen uniform field through a yawed rotor: each element's inflow angle
    follows the skewed-inflow closed form (the advancing and the retreating
    blade see different tangential speeds), alpha = phi - twist_k - pitch
    exactly, and the force splits into q (C_L cos phi + C_D sin phi) along the
    axis and q (C_L sin phi - C_D cos phi) along e_t, nothing radial, with
    C_L, C_D read from an unequally spaced table at that alpha."""
    U, yaw = 0.05, math.radians(yaw_deg)
    a, cl, cd = I.nonuniform_polars()
    pitch = 0.05 if twisted else 0.0
    d = O.make_domain(64, 48, 48, bc=("periodic",) * 3, u_ref=(U, 0, 0))
    t = I.single_turbine(64, 48, 48, diameter=16.0, hub=(20.0, 24.0, 24.0), elements_per_blade=8, yaw=yaw)
    t.update(alpha=a, cl=cl, cd=cd, theta0=0.3, pitch=pitch,
             twist=I.blade_twist(8) if twisted else None)
    s = O.Sim(d, [O.TurbineSpec(**t)])
    s.init_fields()
    step = 3
    pos, fb, alpha, loads = s.alm_forces(s.f, s.falm, step)
    R, ne, Om = t["radius"], t["n_elements"], t["omega"]
    tw = I.blade_twist(8) if twisted else np.zeros(8)
    thrust = torque = 0.0
    for e in range(3 * ne):
        b, k = divmod(e, ne)
        r = (k + 0.5) * R / ne
        theta = 0.3 + Om * step + 2 * math.pi * b / 3
        ea, er, et = _frame(yaw, theta)
        phi, W2 = _skewed_element(U, yaw, Om, r, theta)
        al = phi - tw[k] - pitch
        assert alpha[e] == pytest.approx(al, abs=1e-12)
        CL, CD = np.interp(al, a, cl), np.interp(al, a, cd)
        c = t["chord_root"] + (t["chord_tip"] - t["chord_root"]) * r / R
        q = 0.5 * W2 * c * R / ne
        f_ax, f_t = q * (CL * math.cos(phi) + CD * math.sin(phi)), q * (CL * math.sin(phi) - CD * math.cos(phi))
        np.testing.assert_allclose(fb[e], f_ax * ea + f_t * et, rtol=1e-10, atol=1e-16)
        assert np.dot(fb[e], er) == pytest.approx(0.0, abs=1e-16)
        thrust += f_ax
        torque += r * f_t
    assert loads[0] == pytest.approx(thrust, rel=1e-10)
    assert loads[1] == pytest.approx(torque, rel=1e-10)
    # the same flow with a yaw-free rotor and no twist or pitch gives a different load
    if twisted:
        t0 = dict(t, yaw=0.0, pitch=0.0, twist=None)
        s0 = O.Sim(d, [O.TurbineSpec(**t0)])
        s0.init_fields()
        assert abs(s0.alm_forces(s0.f, s0.falm, step)[3][0] - loads[0]) > 0.05 * abs(loads[0])


def test_unequal_polar_table_is_exact_on_piecewise_linear_data():
    """Linear interpolation in an unequally spaced table reproduces any
    piecewise-linear function whose breakpoints are table nodes, everywhere
    inside the table, and clamps outside; it agrees with numpy's interp."""
    a, cl, cd = I.nonuniform_polars()
    d = np.diff(a)
    assert d.min() < 0.2 * d.max()                      # genuinely unequal spacing
    rng = np.random.default_rng(41)
    xs = np.concatenate([rng.uniform(a[0], a[-1], 400), a[::7], [a[0], a[-1]]])
    for x in xs:
        # C_L is the clipped line, piecewise linear with nodes at the stall corners
        assert O.table_lookup(a, cl, x) == pytest.approx(float(np.clip(2 * math.pi * x, -1.2, 1.2)), abs=1e-13)
        assert O.table_lookup(a, cd, x) == pytest.approx(float(np.interp(x, a, cd)), abs=1e-15)
    for x in (a[0] - 1.0, a[-1] + 0.5):
        assert O.table_lookup(a, cl, x) == (cl[0] if x < a[0] else cl[-1])
    # between two nodes the C_D error is bounded by the spacing: (h^2/8) max|C_D''| = 0.04 h^2/8
    for i in (3, 100, len(a) - 4):
        m = 0.5 * (a[i] + a[i + 1])
        h = a[i + 1] - a[i]
        assert abs(O.table_lookup(a, cd, m) - (0.01 + 0.02 * m * m)) <= 0.04 * h * h / 8 * (1 + 1e-9)
