"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds input data only -- analytic initial fields, seeded random
states, the synthetic rotor and polar tables of the workloads -- and none of the
method's arithmetic (no equilibria, moments, collision or spreading).  Both the
CUDA path and the oracle receive the same arrays from here and turn them into
populations with their own code.

Field layout everywhere: x fastest, arrays shaped (nz, ny, nx); vector fields
(3, nz, ny, nx); non-equilibrium parts (27, nz, ny, nx) in the velocity order
q = (cz+1)*9 + (cy+1)*3 + (cx+1).
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 2402131710


def grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def taylor_green_3d(n, u0, nz=None):
    """3-D Taylor-Green vortex on an n^3 periodic box (k = 2 pi / n):
    u = u0 sin kx cos ky cos kz, v = -u0 cos kx sin ky cos kz, w = 0, and the
    density 1 + 3 p of the incompressible pressure
    p = u0^2/16 (cos 2kx + cos 2ky)(cos 2kz + 2)."""
    nz = n if nz is None else nz
    x, y, z = grid(n, n, nz)
    k = 2 * math.pi / n
    kz = 2 * math.pi / nz
    u = np.stack([u0 * np.sin(k * x) * np.cos(k * y) * np.cos(kz * z),
                  -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(kz * z),
                  np.zeros_like(x)])
    p = u0 ** 2 / 16.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (np.cos(2 * kz * z) + 2.0)
    return 1.0 + 3.0 * p, u


def taylor_green_2d(n, u0, nz=1):
    """z-invariant Taylor-Green vortex (an exact Navier-Stokes solution):
    u = u0 sin kx cos ky, v = -u0 cos kx sin ky, p = -u0^2/4 (cos 2kx + cos 2ky)."""
    x, y, z = grid(n, n, nz)
    k = 2 * math.pi / n
    u = np.stack([u0 * np.sin(k * x) * np.cos(k * y), -u0 * np.cos(k * x) * np.sin(k * y), np.zeros_like(x)])
    p = -u0 ** 2 / 4.0 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    return 1.0 + 3.0 * p, u


def shear_wave(nx, ny, nz, u0, mode=1):
    """u_x = u0 sin(k y), k = 2 pi mode / ny; rho = 1."""
    x, y, z = grid(nx, ny, nz)
    k = 2 * math.pi * mode / ny
    u = np.stack([u0 * np.sin(k * y), np.zeros_like(x), np.zeros_like(x)])
    return np.ones_like(x), u


def random_state(nx, ny, nz, seed=DEFAULT_SEED, u_mean=(0.0, 0.0, 0.0), du=0.02, drho=0.01, fneq_amp=1e-3):
    """Seeded near-equilibrium state: rho = 1 + drho * U(-1,1), u = u_mean + du *
    U(-1,1) per component, and a non-equilibrium perturbation fneq (float32,
    27 planes) of size fneq_amp * scale(class) * U(-1,1), where the class of a
    direction is its number of non-zero velocity components and the scales
    0.3, 0.07, 0.02, 0.005 roughly follow the population sizes."""
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    rho = 1.0 + drho * rng.uniform(-1, 1, shape)
    u = np.stack([u_mean[a] + du * rng.uniform(-1, 1, shape) for a in range(3)])
    # magnitude class per direction: number of non-zero velocity components
    mag = np.array([[0.3, 0.07, 0.02, 0.005][abs(q % 3 - 1) + abs((q // 3) % 3 - 1) + abs(q // 9 - 1)]
                    for q in range(27)])
    fneq = (fneq_amp * mag[:, None, None, None] * rng.uniform(-1, 1, (27,) + shape)).astype(np.float32)
    return rho, u, fneq


# ----------------------------------------------------------------- rotor data

def synthetic_polars(step_deg=0.1, cl_slope=2 * math.pi, cl_max=1.2, cd0=0.01, cd2=0.02):
    """Polar tables of the synthetic rotor: C_L = clip(2 pi alpha, +-1.2),
    C_D = 0.01 + 0.02 alpha^2 (alpha in radians), sampled every step_deg degrees
    over [-180, 180]."""
    n = int(round(360.0 / step_deg)) + 1
    alpha = np.radians(np.linspace(-180.0, 180.0, n))
    cl = np.clip(cl_slope * alpha, -cl_max, cl_max)
    cd = cd0 + cd2 * alpha ** 2
    return alpha, cl, cd


def single_turbine(nx=256, ny=128, nz=128, diameter=32.0, hub=None, elements_per_blade=40, epsilon=2.0,
                   tsr=6.0, u_inf=0.05, chord_root=2.0, chord_tip=1.0, n_blades=3, yaw=0.0, kernel="gauss",
                   tip_loss=False):
    """The single three-bladed rotor of the 256x128x128 actuator-line workload:
    D = 32 cells at (64, 64, 64), 40 elements per blade, eps = 2, TSR 6 at
    U = 0.05, chord 2 -> 1.  Rotor speed omega = TSR U / R (rad per step).
    kernel: force regularisation, "gauss" (width epsilon) or "roma";
    tip_loss: Glauert's tip-loss factor on the element forces."""
    R = diameter / 2.0
    if hub is None:
        hub = (nx / 4.0, ny / 2.0, nz / 2.0)
    alpha, cl, cd = synthetic_polars()
    return dict(hub=tuple(float(h) for h in hub), radius=R, n_blades=n_blades, n_elements=elements_per_blade,
                epsilon=epsilon, omega=tsr * u_inf / R, yaw=yaw, pitch=0.0, theta0=0.0, chord_root=chord_root,
                chord_tip=chord_tip, alpha=alpha, cl=cl, cd=cd, kernel=kernel, tip_loss=tip_loss)


def single_turbine_case(nx=256, ny=128, nz=128, **kw):
    """Domain settings of the single-turbine workload: velocity inlet at x = 0
    (uniform 0.05 with 1 % seeded white noise), zero-gradient outlet,
    periodic y and z, cumulant collision."""
    u_inf = kw.pop("u_inf", 0.05)
    nu = kw.pop("nu", 1e-3)
    seed = kw.pop("seed", DEFAULT_SEED + 2)
    dom = dict(nx=nx, ny=ny, nz=nz, collision="cumulant", nu=nu, smag_c=0.1,
               bc=("inout", "periodic", "periodic"), body_force=(0.0, 0.0, 0.0), inflow_kind=0,
               u_ref=(u_inf, 0.0, 0.0), z0=0.1, z_ref=1.0, noise_rel=0.01, seed=seed)
    turb = single_turbine(nx, ny, nz, u_inf=u_inf, **kw)
    return dom, turb


def batch_instances(n=16, seed=DEFAULT_SEED + 3):
    """Seeded sweep of independent single-turbine instances: domain lengths
    128-384 x 96-160 x 96-160 (multiples of 8), rotor diameters 16-40 cells,
    TSR uniform in [3, 9], inflow 0.03-0.06.  Hub at (nx/4, ny/2, nz/2)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.integers(16, 49)) * 8
        ny = int(rng.integers(12, 21)) * 8
        nz = int(rng.integers(12, 21)) * 8
        d = float(rng.uniform(16, 40))
        d = min(d, 0.5 * min(ny, nz) - 16)   # keep the support inside the domain
        tsr = float(rng.uniform(3, 9))
        u = float(rng.uniform(0.03, 0.06))
        dom, turb = single_turbine_case(nx, ny, nz, diameter=d, tsr=tsr, u_inf=u,
                                        seed=int(rng.integers(0, 2 ** 62)))
        out.append((dom, turb))
    return out


def nonuniform_polars(fine_deg=0.25, coarse_deg=5.0, fine_range_deg=20.0):
    """The synthetic rotor's polars (C_L = clip(2 pi alpha, +-1.2), C_D = 0.01 +
    0.02 alpha^2) tabulated on unequally spaced angles, as real aerofoil tables
    are: every fine_deg degrees on [-fine_range_deg, fine_range_deg], every
    coarse_deg degrees beyond, over [-180, 180], plus the two stall corners
    alpha = +-1.2 / (2 pi)."""
    fine = np.arange(-fine_range_deg, fine_range_deg + 0.5 * fine_deg, fine_deg)
    coarse = np.arange(-180.0, 180.0 + 0.5 * coarse_deg, coarse_deg)
    coarse = coarse[np.abs(coarse) > fine_range_deg]
    stall = np.degrees([-1.2 / (2 * math.pi), 1.2 / (2 * math.pi)])
    deg = np.unique(np.round(np.concatenate([fine, coarse, stall]), 12))
    alpha = np.radians(deg)
    cl = np.clip(2 * math.pi * alpha, -1.2, 1.2)
    cd = 0.01 + 0.02 * alpha ** 2
    return alpha, cl, cd


def blade_twist(n_elements, root=0.20, tip=0.02):
    """Twist of element k (radians), linear from `root` at the blade root to
    `tip` at the tip, at the element centres r_k = (k + 1/2) R / N_e."""
    s = (np.arange(n_elements) + 0.5) / n_elements
    return root + (tip - root) * s


def yawed_twisted_rotor(nx=64, ny=40, nz=40, diameter=16.0, elements_per_blade=8, yaw_deg=7.0, pitch=0.05,
                        seed=778, **kw):
    """The scaled-down single-rotor case with every blade-geometry option on:
    yaw yaw_deg degrees, a twist table, a collective pitch, and polars on
    unequally spaced angles (nonuniform_polars)."""
    dom, turb = single_turbine_case(nx, ny, nz, diameter=diameter, elements_per_blade=elements_per_blade, seed=seed,
                                    yaw=math.radians(yaw_deg), **kw)
    alpha, cl, cd = nonuniform_polars()
    turb.update(alpha=alpha, cl=cl, cd=cd, pitch=float(pitch), twist=blade_twist(elements_per_blade),
                theta0=0.3)
    return dom, turb


def log_law_profile(nz, u_hub, z0, z_hub):
    """Mean streamwise inflow u(z) = u_hub ln(z_c / z0) / ln(z_hub / z0) at the
    cell centres z_c = z + 1/2 above the bottom face."""
    zc = np.arange(nz) + 0.5
    return u_hub * np.log(zc / z0) / math.log(z_hub / z0)


def small_farm_case(nx=96, ny=48, nz=40, diameter=12.0, elements_per_blade=6, u_hub=0.05, tsr=6.0,
                    yaw_deg=(5.0, 9.0), x_hubs=(20.0, 60.0), seed=2402131715):
    """A scaled-down version of the 3x3 farm: log-law inflow (z0 = 0.1, hub
    height z_ref = nz / 2) with 1 % noise at the x inlet, zero-gradient outlet,
    periodic y, free-slip bottom and top, and two yawed rotors in a row
    (x_hubs, at mid-span and hub height)."""
    z_hub = nz / 2.0
    dom = dict(nx=nx, ny=ny, nz=nz, collision="cumulant", nu=1e-3, smag_c=0.1,
               bc=("inout", "periodic", "freeslip"), body_force=(0.0, 0.0, 0.0), inflow_kind=1,
               u_ref=(u_hub, 0.0, 0.0), z0=0.1, z_ref=z_hub, noise_rel=0.01, seed=seed)
    turbs = []
    for xh, yd in zip(x_hubs, yaw_deg):
        turbs.append(single_turbine(nx, ny, nz, diameter=diameter, hub=(xh, ny / 2.0, z_hub),
                                    elements_per_blade=elements_per_blade, tsr=tsr, u_inf=u_hub,
                                    yaw=math.radians(yd)))
    return dom, turbs
