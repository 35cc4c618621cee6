"""Pins of the oracle's single-cell algebra against definitions and closed forms.

Each test checks the oracle against something other than itself: the defining
sums written out by brute force, the moment generating series of the
cumulants, the BGK limit of the cumulant operator, exact conservation, and the
published splitmix64 output.
"""
import math

import numpy as np
import pytest

import oracle as O

C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], dtype=np.float64)
MIDX = [(m % 3, (m // 3) % 3, m // 9) for m in range(27)]


def rand_f(rng, u=(0.04, -0.03, 0.02), amp=0.02):
    f = O.equilibrium(1.0 + 0.05 * rng.uniform(-1, 1), u)
    return f * (1.0 + amp * rng.uniform(-1, 1, 27))


def brute_central(f, u):
    return np.array([np.sum((C[:, 0] - u[0]) ** a * (C[:, 1] - u[1]) ** b * (C[:, 2] - u[2]) ** c * f)
                     for (a, b, c) in MIDX])


# ------------------------------------------------------------- moments

def test_central_moments_match_definition():
    rng = np.random.default_rng(1)
    for _ in range(5):
        f = rng.uniform(0.001, 0.3, 27)
        u = rng.uniform(-0.1, 0.1, 3)
        np.testing.assert_allclose(O.central_moments(f, u), brute_central(f, u), rtol=0, atol=1e-15)


def test_population_round_trip_is_identity():
    rng = np.random.default_rng(2)
    for _ in range(5):
        f = rng.uniform(0.001, 0.3, 27)
        u = rng.uniform(-0.2, 0.2, 3)
        np.testing.assert_allclose(O.populations_from_central(O.central_moments(f, u), u), f, atol=1e-14)


def test_equilibrium_moments():
    """Product equilibrium: mass rho, momentum rho u, central second moments
    rho/3 on the diagonal and 0 off it, and it is separable per axis."""
    rho, u = 1.07, np.array([0.05, -0.02, 0.03])
    f = O.equilibrium(rho, u)
    k = brute_central(f, u)
    assert abs(f.sum() - rho) < 1e-15
    np.testing.assert_allclose(C.T @ f, rho * u, atol=1e-15)
    for m, (a, b, c) in enumerate(MIDX):
        # central moments of a product measure factorise: rho * prod k1d(order)
        k1d = {0: 1.0, 1: 0.0, 2: 1.0 / 3.0}
        assert abs(k[m] - rho * k1d[a] * k1d[b] * k1d[c]) < 1e-15, (a, b, c)
    # u = 0: the lattice weights 8/27, 2/27, 1/54, 1/216
    w = O.equilibrium(1.0, [0, 0, 0])
    cls = np.abs(C).sum(1).astype(int)
    for n, val in enumerate([8 / 27, 2 / 27, 1 / 54, 1 / 216]):
        np.testing.assert_allclose(w[cls == n], val, atol=1e-17)


def test_poly_equilibrium_moments():
    """Polynomial equilibrium: mass, momentum and momentum flux rho/3 I + rho u u."""
    rho, u = 0.98, np.array([0.03, 0.01, -0.04])
    f = O.equilibrium_poly(rho, u)
    assert abs(f.sum() - rho) < 1e-15
    np.testing.assert_allclose(C.T @ f, rho * u, atol=1e-15)
    Pi = np.einsum("qa,qb,q->ab", C, C, f)
    np.testing.assert_allclose(Pi, rho / 3 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)


# ------------------------------------------------------------- cumulants

def _poly_mul(P, Q):
    """Product of two series truncated at degree 2 in each of three variables."""
    R = np.zeros((3, 3, 3))
    for a1 in range(3):
        for b1 in range(3):
            for c1 in range(3):
                if P[a1, b1, c1] == 0:
                    continue
                for a2 in range(3 - a1):
                    for b2 in range(3 - b1):
                        for c2 in range(3 - c1):
                            R[a1 + a2, b1 + b2, c1 + c2] += P[a1, b1, c1] * Q[a2, b2, c2]
    return R


def cumulants_by_log_series(kappa):
    """Cumulants as the Taylor coefficients of K(t) = ln M(t), M the moment
    generating series of the normalised central moments (first order set to 0).
    Truncating each variable at degree 2 is exact for the coefficients kept."""
    rho = kappa[0]
    M = np.zeros((3, 3, 3))
    for m, (a, b, c) in enumerate(MIDX):
        if a + b + c == 1:
            continue
        M[a, b, c] = kappa[m] / rho / (math.factorial(a) * math.factorial(b) * math.factorial(c))
    X = M.copy()
    X[0, 0, 0] = 0.0
    K = np.zeros((3, 3, 3))
    P = np.zeros((3, 3, 3))
    P[0, 0, 0] = 1.0
    for n in range(1, 7):
        P = _poly_mul(P, X)
        K += (-1) ** (n + 1) * P / n
    out = np.zeros(27)
    for m, (a, b, c) in enumerate(MIDX):
        out[m] = rho * K[a, b, c] * math.factorial(a) * math.factorial(b) * math.factorial(c)
    return out


def test_cumulants_match_log_series():
    rng = np.random.default_rng(3)
    for trial in range(4):
        f = rng.uniform(0.005, 0.2, 27)
        rho = f.sum()
        u = C.T @ f / rho
        k = O.central_moments(f, u)
        Cum = O.cumulants_from_central(k)
        ref = cumulants_by_log_series(k)
        for m, (a, b, c) in enumerate(MIDX):
            if a + b + c >= 2:
                assert abs(Cum[m] - ref[m]) < 1e-14, (trial, (a, b, c), Cum[m], ref[m])
        assert Cum[0] == pytest.approx(rho, abs=1e-15)


def test_cumulant_round_trip_and_gaussian_closure():
    rng = np.random.default_rng(4)
    f = rng.uniform(0.005, 0.2, 27)
    u = C.T @ f / f.sum()
    k = O.central_moments(f, u)
    k2 = O.central_from_cumulants(O.cumulants_from_central(k))
    np.testing.assert_allclose(k2, k, atol=1e-15)
    # cumulants vanish above order 2  <=>  moments are Isserlis products
    Cg = np.zeros(27)
    Cg[0] = 1.3
    S = {(2, 0, 0): 0.4, (0, 2, 0): 0.35, (0, 0, 2): 0.3, (1, 1, 0): 0.02, (1, 0, 1): -0.01, (0, 1, 1): 0.03}
    for m, idx in enumerate(MIDX):
        if idx in S:
            Cg[m] = 1.3 * S[idx]
    kg = O.central_from_cumulants(Cg) / 1.3
    sxx, syy, szz, sxy, sxz, syz = S[(2, 0, 0)], S[(0, 2, 0)], S[(0, 0, 2)], S[(1, 1, 0)], S[(1, 0, 1)], S[(0, 1, 1)]
    iss = sxx * syy * szz + 2 * sxx * syz ** 2 + 2 * syy * sxz ** 2 + 2 * szz * sxy ** 2 + 8 * sxy * sxz * syz
    assert kg[MIDX.index((2, 2, 2))] == pytest.approx(iss, abs=1e-15)
    assert kg[MIDX.index((2, 1, 1))] == pytest.approx(sxx * syz + 2 * sxy * sxz, abs=1e-15)
    assert kg[MIDX.index((1, 2, 2))] == pytest.approx(0.0, abs=1e-15)
    assert O.partition_term_count() == 18 + 30 + 40


# ------------------------------------------------------------- collisions

PROD = lambda w: [w] + [1.0] * 9  # production rates: shear omega, all others 1


def test_equilibrium_is_fixed_point():
    for u in ([0, 0, 0], [0.05, -0.03, 0.02]):
        feq = O.equilibrium(1.02, u)
        for w in (0.7, 1.3, 1.95):
            np.testing.assert_allclose(O.collide_cumulant(feq, [0, 0, 0], PROD(w)), feq, atol=2e-16)


def test_all_rates_one_gives_equilibrium():
    rng = np.random.default_rng(5)
    f = rand_f(rng, amp=0.2)
    rho = f.sum()
    u = C.T @ f / rho
    np.testing.assert_allclose(O.collide_cumulant(f, [0, 0, 0], [1.0] * 10), O.equilibrium(rho, u), atol=1e-16)


def test_conservation_both_operators():
    rng = np.random.default_rng(6)
    for _ in range(5):
        f = rand_f(rng, amp=0.1)
        F = rng.uniform(-1e-3, 1e-3, 3)
        for out in (O.collide_cumulant(f, F, PROD(1.7)),
                    O.collide_cumulant(f, F, list(rng.uniform(0.5, 1.9, 10))),
                    O.collide_srt_smag(f, F, 0.01, 0.15)):
            assert abs(out.sum() - f.sum()) < 1e-15
            np.testing.assert_allclose(C.T @ out, C.T @ f + F, atol=1e-16)


def test_small_perturbation_equals_bgk():
    """With every rate = omega the cumulant operator is BGK(omega) toward the
    product equilibrium up to O(delta^2) in the non-equilibrium amplitude."""
    rng = np.random.default_rng(7)
    u = np.array([0.03, -0.02, 0.01])
    g = rng.uniform(-1, 1, 27)
    g -= g.mean()
    omega = 1.3
    diffs = []
    for delta in (1e-3, 5e-4, 2.5e-4):
        f = O.equilibrium(1.0, u) + delta * g * O.equilibrium(1.0, [0, 0, 0])
        rho = f.sum()
        uu = C.T @ f / rho
        bgk = f + omega * (O.equilibrium(rho, uu) - f)
        diffs.append(np.abs(O.collide_cumulant(f, [0, 0, 0], [omega] * 10) - bgk).max())
    assert diffs[0] < 1e-5
    # quadratic convergence
    assert diffs[0] / diffs[1] == pytest.approx(4.0, rel=0.1)
    assert diffs[1] / diffs[2] == pytest.approx(4.0, rel=0.1)


def test_shear_relaxation_acts_only_on_deviatoric_second_order():
    """Relaxing with production rates: post-collision second central moments are
    rho/3 I + (1-omega) * (deviatoric part), the trace goes to rho."""
    rng = np.random.default_rng(8)
    f = rand_f(rng, amp=0.1)
    rho = f.sum()
    u = C.T @ f / rho
    w = 1.6
    out = O.collide_cumulant(f, [0, 0, 0], PROD(w))
    u2 = C.T @ out / rho
    np.testing.assert_allclose(u2, u, atol=1e-16)
    k_in = brute_central(f, u)
    k_out = brute_central(out, u)
    ii = {n: MIDX.index(n) for n in [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]}
    T_in = sum(k_in[ii[n]] for n in [(2, 0, 0), (0, 2, 0), (0, 0, 2)])
    T_out = sum(k_out[ii[n]] for n in [(2, 0, 0), (0, 2, 0), (0, 0, 2)])
    assert T_out == pytest.approx(rho, abs=1e-15)
    for n in [(1, 1, 0), (1, 0, 1), (0, 1, 1)]:
        assert k_out[ii[n]] == pytest.approx((1 - w) * k_in[ii[n]], abs=1e-15)
    d_in = k_in[ii[(2, 0, 0)]] - k_in[ii[(0, 2, 0)]]
    d_out = k_out[ii[(2, 0, 0)]] - k_out[ii[(0, 2, 0)]]
    assert d_out == pytest.approx((1 - w) * d_in, abs=1e-15)
    # all third-order central moments vanish after full relaxation
    for m, (a, b, c) in enumerate(MIDX):
        if a + b + c == 3:
            assert abs(k_out[m]) < 1e-15


def test_srt_without_smagorinsky_is_bgk_guo():
    rng = np.random.default_rng(9)
    f = rand_f(rng, amp=0.05)
    F = np.array([1e-4, -2e-4, 5e-5])
    nu = 0.02
    om = O.omega_from_nu(nu)
    assert om == pytest.approx(1.0 / (3 * nu + 0.5))
    rho = f.sum()
    u = (C.T @ f + F / 2) / rho
    feq = O.equilibrium_poly(rho, u)
    w = O.equilibrium(1.0, [0, 0, 0])
    cu = C @ u
    S = (1 - om / 2) * w * ((3 * (C - u) + 9 * cu[:, None] * C) @ F)
    np.testing.assert_allclose(O.collide_srt_smag(f, F, nu, 0.0), f - om * (f - feq) + S, atol=1e-17)


def test_smagorinsky_increases_effective_viscosity():
    """With C > 0 the operator relaxes like BGK with omega_eff < omega0, where
    tau_eff = 1/omega_eff solves tau^2 - tau0 tau - 9 sqrt(2) C^2 |Pi|/(2 rho) = 0."""
    rng = np.random.default_rng(10)
    f = rand_f(rng, amp=0.1)
    nu, Cs = 0.01, 0.2
    out0 = O.collide_srt_smag(f, [0, 0, 0], nu, 0.0)
    out1 = O.collide_srt_smag(f, [0, 0, 0], nu, Cs)
    rho = f.sum()
    u = C.T @ f / rho
    feq = O.equilibrium_poly(rho, u)
    # recover omega_eff from the relaxation of the non-equilibrium part
    neq = f - feq
    om_eff = np.dot(f - out1, neq) / np.dot(neq, neq)
    om0 = np.dot(f - out0, neq) / np.dot(neq, neq)
    assert om0 == pytest.approx(O.omega_from_nu(nu), rel=1e-12)
    Pi = np.einsum("qa,qb,q->ab", C, C, neq)
    tau, tau0 = 1 / om_eff, 1 / om0
    assert tau * tau - tau0 * tau == pytest.approx(9 * math.sqrt(2) * Cs ** 2 * np.linalg.norm(Pi) / (2 * rho), rel=1e-10)


# ------------------------------------------------------------- rng

def test_splitmix64_published_value():
    # first output of splitmix64 with state 0 (Vigna's reference implementation)
    assert O.splitmix64(0, 1) == 0xE220A8397B1DCDAF
    assert O.splitmix64(0, 2) == 0x6E789E6AA1B965F4


def test_inflow_noise_statistics():
    d = O.make_domain(8, 64, 64, bc=("inout", "periodic", "periodic"), u_ref=(0.05, 0, 0), noise_rel=0.01,
                      seed=1234)
    us = np.array([O.inflow_velocity(d, n, y, z) for n in range(4) for y in range(0, 64, 3) for z in range(0, 64, 5)])
    dev = us - np.array([0.05, 0, 0])
    assert np.abs(dev).max() <= 0.01 * 0.05 + 1e-15
    assert abs(dev.mean()) < 1e-4 * 0.05 * 10
    # uniform on [-a, a): variance a^2/3
    assert dev.var() == pytest.approx((0.0005 ** 2) / 3, rel=0.1)
    # different steps give different noise, same step is reproducible
    assert not np.allclose(O.inflow_velocity(d, 0, 1, 1), O.inflow_velocity(d, 1, 1, 1))
    np.testing.assert_array_equal(O.inflow_velocity(d, 5, 3, 2), O.inflow_velocity(d, 5, 3, 2))
