"""FP64 CPU oracle for the D3Q27 cumulant LBM + actuator line (arxiv 2402.13171).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow restatement of the
method in C (``lbm_oracle.c``) with this thin ctypes wrapper.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py`` may import
it; the product package never does, and the two share no code.

Parity status of each function (what pins it; see tests/test_oracle_*.py):
  equilibrium, macroscopic, central moments ....... brute-force definition, closed forms
  cumulants <-> central moments ................... log of the moment generating series
  cumulant collision .............................. fixed point, omega=1, BGK limit, conservation,
                                                    shear-wave / Taylor-Green decay
  SRT-Smagorinsky collision ....................... C=0 -> plain BGK-Guo conservation,
                                                    Poiseuille closed form, eddy-viscosity closed form
  pull streaming + boundaries ..................... periodic shift, bounce-back Poiseuille,
                                                    inlet/outlet constant-state invariance
  blade kinematics, sampling, element forces ...... frozen-field closed form, affine exactness
  Glauert tip-loss factor ......................... closed-form values, limits, frozen-field loads
  Gaussian spreading .............................. force-sum, separable closed form
  Roma discrete-delta spreading ................... Roma's three moment conditions, force-sum,
                                                    force centroid at the element
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

NQ = 27


def build(force: bool = False) -> str:
    """Compile the C oracle into a shared library (gcc, OpenMP, -O2, no fast-math)."""
    import platform
    os.makedirs(_BUILD, exist_ok=True)
    stamp = os.path.join(_BUILD, "ARCH")
    if (open(stamp).read().strip() if os.path.exists(stamp) else "") != platform.machine():
        force = True
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    with open(stamp, "w") as f:
        f.write(platform.machine())
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


class Domain(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("nu", ctypes.c_double), ("smag_c", ctypes.c_double),
        ("bc", ctypes.c_int * 3),
        ("body_force", ctypes.c_double * 3),
        ("inflow_kind", ctypes.c_int),
        ("u_ref", ctypes.c_double * 3),
        ("z0", ctypes.c_double), ("z_ref", ctypes.c_double),
        ("noise_rel", ctypes.c_double),
        ("seed", ctypes.c_ulonglong),
    ]


class Turbine(ctypes.Structure):
    _fields_ = [
        ("hub", ctypes.c_double * 3),
        ("radius", ctypes.c_double),
        ("n_blades", ctypes.c_int), ("n_elements", ctypes.c_int),
        ("epsilon", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("yaw", ctypes.c_double), ("pitch", ctypes.c_double), ("theta0", ctypes.c_double),
        ("chord_root", ctypes.c_double), ("chord_tip", ctypes.c_double),
        ("twist", _dp),
        ("n_polar", ctypes.c_int),
        ("alpha", _dp), ("cl", _dp), ("cd", _dp),
        ("kernel", ctypes.c_int),
        ("tip_loss", ctypes.c_int),
    ]


def _declare(L):
    c_long = ctypes.c_long
    L.or_num_threads.restype = ctypes.c_int
    L.or_set_num_threads.argtypes = [ctypes.c_int]
    L.or_equilibrium.argtypes = [ctypes.c_double, _dp, _dp]
    L.or_equilibrium_poly.argtypes = [ctypes.c_double, _dp, _dp]
    L.or_macroscopic.argtypes = [_dp, _dp, _dp, _dp]
    L.or_central_moments.argtypes = [_dp, _dp, _dp]
    L.or_populations_from_central.argtypes = [_dp, _dp, _dp]
    L.or_cumulants_from_central.argtypes = [_dp, _dp]
    L.or_central_from_cumulants.argtypes = [_dp, _dp]
    L.or_partition_term_count.restype = ctypes.c_int
    L.or_collide_cumulant.argtypes = [_dp, _dp, _dp, _dp]
    L.or_collide_srt_smag.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
    L.or_omega_from_nu.argtypes = [ctypes.c_double]
    L.or_omega_from_nu.restype = ctypes.c_double
    L.or_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    L.or_splitmix64.restype = ctypes.c_uint64
    L.or_inflow_velocity.argtypes = [ctypes.POINTER(Domain), c_long, ctypes.c_int, ctypes.c_int, _dp]
    L.or_pull_cell.argtypes = [ctypes.POINTER(Domain), _dp, c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    L.or_element_kinematics.argtypes = [ctypes.POINTER(Turbine), c_long, ctypes.c_int, ctypes.c_int,
                                        _dp, _dp, _dp, _dp, _dp, _dp]
    L.or_table_lookup.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double]
    L.or_table_lookup.restype = ctypes.c_double
    L.or_sample.argtypes = [ctypes.POINTER(Domain), _dp, _dp, c_long, _dp, _dp, _dp]
    L.or_alm_forces.argtypes = [ctypes.POINTER(Domain), ctypes.POINTER(Turbine), _dp, _dp, c_long, _dp, _dp, _dp, _dp]
    L.or_gauss_axis_sum.argtypes = [ctypes.c_double, ctypes.c_double]
    L.or_gauss_axis_sum.restype = ctypes.c_double
    L.or_spread.argtypes = [ctypes.POINTER(Domain), _dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]
    L.or_spread_at.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, _dp]
    L.or_roma_phi.argtypes = [ctypes.c_double]
    L.or_roma_phi.restype = ctypes.c_double
    L.or_tip_loss.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.or_tip_loss.restype = ctypes.c_double
    L.or_step.argtypes = [ctypes.POINTER(Domain), ctypes.POINTER(Turbine), ctypes.c_int, _dp, _dp, _dp, _dp, c_long,
                          _dp, _dp, _dp]
    L.or_step_planes.argtypes = [ctypes.POINTER(Domain), ctypes.POINTER(Turbine), ctypes.c_int, _dp, _dp, _dp, _dp,
                                 c_long, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int]
    L.or_update_cell.argtypes = [ctypes.POINTER(Domain), _dp, _dp, c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    L.or_moments.argtypes = [ctypes.POINTER(Domain), _dp, _dp, _dp, _dp]
    L.or_init_fields.argtypes = [ctypes.POINTER(Domain), _dp, _dp, _fp, _dp]


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _d(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.shape, n)
    return a


# ---------------------------------------------------------------- single cell

def equilibrium(rho, u):
    out = np.zeros(NQ)
    lib().or_equilibrium(float(rho), _p(_d(u, 3)), _p(out))
    return out


def equilibrium_poly(rho, u):
    out = np.zeros(NQ)
    lib().or_equilibrium_poly(float(rho), _p(_d(u, 3)), _p(out))
    return out


def macroscopic(f, F=(0, 0, 0)):
    rho = np.zeros(1)
    u = np.zeros(3)
    lib().or_macroscopic(_p(_d(f, NQ)), _p(_d(F, 3)), _p(rho), _p(u))
    return rho[0], u


def central_moments(f, u):
    out = np.zeros(NQ)
    lib().or_central_moments(_p(_d(f, NQ)), _p(_d(u, 3)), _p(out))
    return out


def populations_from_central(k, u):
    out = np.zeros(NQ)
    lib().or_populations_from_central(_p(_d(k, NQ)), _p(_d(u, 3)), _p(out))
    return out


def cumulants_from_central(k):
    out = np.zeros(NQ)
    lib().or_cumulants_from_central(_p(_d(k, NQ)), _p(out))
    return out


def central_from_cumulants(C):
    out = np.zeros(NQ)
    lib().or_central_from_cumulants(_p(_d(C, NQ)), _p(out))
    return out


def partition_term_count():
    return lib().or_partition_term_count()


def collide_cumulant(f, F, rates):
    out = np.zeros(NQ)
    lib().or_collide_cumulant(_p(_d(f, NQ)), _p(_d(F, 3)), _p(_d(rates, 10)), _p(out))
    return out


def collide_srt_smag(f, F, nu, smag_c):
    out = np.zeros(NQ)
    lib().or_collide_srt_smag(_p(_d(f, NQ)), _p(_d(F, 3)), float(nu), float(smag_c), _p(out))
    return out


def omega_from_nu(nu):
    return lib().or_omega_from_nu(float(nu))


def splitmix64(seed, k):
    return int(lib().or_splitmix64(ctypes.c_uint64(seed), ctypes.c_uint64(k)))


def table_lookup(xs, ys, x):
    xs = _d(xs)
    ys = _d(ys)
    return lib().or_table_lookup(_p(xs), _p(ys), xs.size, float(x))


def gauss_axis_sum(p, eps):
    return lib().or_gauss_axis_sum(float(p), float(eps))


KERNEL = {"gauss": 0, "roma": 1}


def roma_phi(r):
    """Roma et al.'s three-point discrete delta at r (Sec. 2.2)."""
    return lib().or_roma_phi(float(r))


def tip_loss(n_blades, R, r, phi):
    """Glauert's tip-loss factor (Prandtl's form) of an element (Sec. 2.2)."""
    return lib().or_tip_loss(int(n_blades), float(R), float(r), float(phi))


# ---------------------------------------------------------------- domain

BC = {"periodic": 0, "inout": 1, "noslip": 2, "freeslip": 3}
COLL = {"cumulant": 0, "srt_smag": 1}


def make_domain(nx, ny, nz, collision="cumulant", nu=0.01, smag_c=0.0, bc=("periodic",) * 3,
                body_force=(0, 0, 0), inflow_kind=0, u_ref=(0, 0, 0), z0=0.1, z_ref=1.0, noise_rel=0.0,
                seed=0) -> Domain:
    d = Domain()
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    d.collision = COLL[collision] if isinstance(collision, str) else int(collision)
    d.nu = float(nu)
    d.smag_c = float(smag_c)
    for a in range(3):
        d.bc[a] = BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
        d.body_force[a] = float(body_force[a])
        d.u_ref[a] = float(u_ref[a])
    d.inflow_kind = int(inflow_kind)
    d.z0 = float(z0)
    d.z_ref = float(z_ref)
    d.noise_rel = float(noise_rel)
    d.seed = int(seed) & ((1 << 64) - 1)
    return d


class TurbineSpec:
    """Owns the numpy arrays an oracle Turbine struct points into."""

    def __init__(self, hub, radius, n_blades, n_elements, epsilon, omega, alpha, cl, cd, yaw=0.0, pitch=0.0,
                 theta0=0.0, chord_root=1.0, chord_tip=1.0, twist=None, kernel="gauss", tip_loss=False):
        self.alpha = _d(alpha)
        self.cl = _d(cl)
        self.cd = _d(cd)
        self.twist = None if twist is None else _d(twist, n_elements)
        t = Turbine()
        for a in range(3):
            t.hub[a] = float(hub[a])
        t.radius = float(radius)
        t.n_blades = int(n_blades)
        t.n_elements = int(n_elements)
        t.epsilon = float(epsilon)
        t.omega = float(omega)
        t.yaw = float(yaw)
        t.pitch = float(pitch)
        t.theta0 = float(theta0)
        t.chord_root = float(chord_root)
        t.chord_tip = float(chord_tip)
        t.twist = _p(self.twist)
        t.n_polar = self.alpha.size
        t.alpha = _p(self.alpha)
        t.cl = _p(self.cl)
        t.cd = _p(self.cd)
        t.kernel = KERNEL[kernel]
        t.tip_loss = int(bool(tip_loss))
        self.struct = t

    @property
    def n_el(self):
        return self.struct.n_blades * self.struct.n_elements


def inflow_velocity(dom, step, y, z):
    u = np.zeros(3)
    lib().or_inflow_velocity(ctypes.byref(dom), int(step), int(y), int(z), _p(u))
    return u


def element_kinematics(turb: TurbineSpec, step, b, k):
    out = [np.zeros(3) for _ in range(5)]
    r = np.zeros(1)
    lib().or_element_kinematics(ctypes.byref(turb.struct), int(step), int(b), int(k), *[_p(o) for o in out], _p(r))
    pos, vel, ea, er, et = out
    return dict(pos=pos, vel=vel, e_axis=ea, e_r=er, e_t=et, r=r[0])


class Sim:
    """A whole-domain oracle run: f (27, nz, ny, nx) float64, q-major."""

    def __init__(self, dom: Domain, turbines=()):
        self.dom = dom
        self.turbines = list(turbines)
        self.N = dom.nx * dom.ny * dom.nz
        shape = (NQ, dom.nz, dom.ny, dom.nx)
        self.f = np.zeros(shape)
        self.g = np.zeros(shape)
        self.falm = np.zeros((3, dom.nz, dom.ny, dom.nx))
        self.falm_next = np.zeros_like(self.falm)
        self.step_count = 0
        n_t = max(1, len(self.turbines))
        self.loads = np.zeros((n_t, 2))
        n_el = sum(t.n_el for t in self.turbines)
        self.elem_pos = np.zeros((max(n_el, 1), 3))
        self.elem_force = np.zeros((max(n_el, 1), 3))
        arr = (Turbine * n_t)()
        for i, t in enumerate(self.turbines):
            arr[i] = t.struct
        self._tarr = arr

    def init_fields(self, rho=None, u=None, fneq=None):
        N = self.N
        if rho is None:
            rho = np.ones(N)
        if u is None:
            # the mean inflow everywhere: uniform u_ref, or u_ref scaled by the
            # log law ln(z_c/z0)/ln(z_ref/z0) at the cell-centre height z_c = z + 1/2
            d = self.dom
            scale = np.ones(d.nz)
            if d.inflow_kind == 1:
                scale = np.log((np.arange(d.nz) + 0.5) / d.z0) / np.log(d.z_ref / d.z0)
            u = np.zeros((3, d.nz, d.ny * d.nx))
            for a in range(3):
                u[a] = d.u_ref[a] * scale[:, None]
            u = u.reshape(3, N)
        rho = _d(rho, N)
        u = _d(u, 3 * N)
        fn = None
        if fneq is not None:
            fn = np.ascontiguousarray(np.asarray(fneq, dtype=np.float32))
            assert fn.size == NQ * N
        lib().or_init_fields(ctypes.byref(self.dom), _p(rho), _p(u),
                             fn.ctypes.data_as(_fp) if fn is not None else None, _p(self.f))
        self.falm[:] = 0
        self.step_count = 0

    def step(self, n=1):
        for _ in range(n):
            lib().or_step(ctypes.byref(self.dom), self._tarr, len(self.turbines), _p(self.f), _p(self.g),
                          _p(self.falm), _p(self.falm_next), self.step_count, _p(self.loads), _p(self.elem_pos),
                          _p(self.elem_force))
            self.f, self.g = self.g, self.f
            self.falm, self.falm_next = self.falm_next, self.falm
            self.step_count += 1

    def step_planes(self, z_begin, z_end):
        """One step whose stream-collide part covers planes [z_begin, z_end) only
        (a bounded CPU-timing sample; the state outside is not advanced)."""
        lib().or_step_planes(ctypes.byref(self.dom), self._tarr, len(self.turbines), _p(self.f), _p(self.g),
                             _p(self.falm), _p(self.falm_next), self.step_count, _p(self.loads), _p(self.elem_pos),
                             _p(self.elem_force), int(z_begin), int(z_end))
        self.f, self.g = self.g, self.f
        self.falm, self.falm_next = self.falm_next, self.falm
        self.step_count += 1

    def moments(self):
        rho = np.zeros((self.dom.nz, self.dom.ny, self.dom.nx))
        u = np.zeros((3, self.dom.nz, self.dom.ny, self.dom.nx))
        lib().or_moments(ctypes.byref(self.dom), _p(self.f), _p(self.falm), _p(rho), _p(u))
        return rho, u

    # single-cell helpers on an arbitrary source array (for sampled checks)
    def pull_cell(self, fsrc, step, x, y, z):
        out = np.zeros(NQ)
        lib().or_pull_cell(ctypes.byref(self.dom), _p(fsrc), int(step), int(x), int(y), int(z), _p(out))
        return out

    def update_cell(self, fsrc, F, step, x, y, z):
        out = np.zeros(NQ)
        lib().or_update_cell(ctypes.byref(self.dom), _p(fsrc), _p(_d(F, 3)), int(step), int(x), int(y), int(z),
                             _p(out))
        return out

    def alm_forces(self, fsrc, falm_prev, step, turbine_index=0):
        t = self.turbines[turbine_index]
        ne = t.n_el
        pos = np.zeros((ne, 3))
        fb = np.zeros((ne, 3))
        alpha = np.zeros(ne)
        loads = np.zeros(2)
        lib().or_alm_forces(ctypes.byref(self.dom), ctypes.byref(t.struct), _p(fsrc), _p(falm_prev), int(step),
                            _p(pos), _p(fb), _p(alpha), _p(loads))
        return pos, fb, alpha, loads

    def sample(self, fsrc, falm_prev, step, p):
        rho = np.zeros(1)
        u = np.zeros(3)
        lib().or_sample(ctypes.byref(self.dom), _p(fsrc), _p(falm_prev), int(step), _p(_d(p, 3)), _p(rho), _p(u))
        return rho[0], u


def spread(dom, pos, fblade, eps, kernel="gauss"):
    pos = _d(pos)
    fb = _d(fblade)
    force = np.zeros((3, dom.nz, dom.ny, dom.nx))
    lib().or_spread(ctypes.byref(dom), _p(pos), _p(fb), pos.size // 3, float(eps), KERNEL[kernel], _p(force))
    return force


def spread_at(pos, fblade, eps, x, y, z, kernel="gauss"):
    pos = _d(pos)
    fb = _d(fblade)
    out = np.zeros(3)
    lib().or_spread_at(_p(pos), _p(fb), pos.size // 3, float(eps), KERNEL[kernel], int(x), int(y), int(z),
                       _p(out))
    return out


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    lib().or_set_num_threads(int(n))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
