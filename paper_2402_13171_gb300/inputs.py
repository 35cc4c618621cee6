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
