"""Learned warm start: a wake surrogate trained on this solver's own mean wakes.

Binding of the mlp_* calls of include/lbm_gb300.h (forward, loss gradient and
Adam training run in the CUDA library) plus the host logic around it:

* ``generate_wake_data``: single-rotor lattice runs with seeded (TSR, yaw,
  U_hub) whose time-mean velocity is probed on a grid behind the rotor;
* features (x/D, y/D, z/D relative to the hub, TSR, yaw, U_hub), scaled to
  O(1), and targets (u/U - 1, v/U, w/U);
* ``farm_initial_velocity``: for a farm, each rotor's predicted wake on a
  coarse grid, combined by summing squared velocity deficits (Katic et al.
  1986) on the inflow profile and repeated to cell resolution;
* ``WindowMeans`` / ``settle_step``: window means of u_x on a plane and the
  first window within a tolerance of the converged mean (the mean of a long
  run's second half; the tolerance is a multiple of that run's noise floor).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import lbm

_fp = ctypes.POINTER(ctypes.c_float)
_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    L = lbm.load()
    if getattr(L, "_mlp_declared", False):
        return L
    vp = ctypes.c_void_p
    L.mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.mlp_destroy.argtypes = [vp]
    L.mlp_destroy.restype = None
    L.mlp_last_error.argtypes = [vp]
    L.mlp_last_error.restype = ctypes.c_char_p
    L.mlp_num_params.argtypes = [vp]
    L.mlp_num_params.restype = ctypes.c_int
    for name, args in {"mlp_set_params": [vp, _fp], "mlp_get_params": [vp, _fp],
                       "mlp_forward": [vp, _fp, ctypes.c_int, _fp],
                       "mlp_loss_grad": [vp, _fp, _fp, ctypes.c_int, _dp, _fp],
                       "mlp_set_data": [vp, _fp, _fp, ctypes.c_int],
                       "mlp_train": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong, _dp]}.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L._mlp_declared = True
    return L


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class WakeMLP:
    """n_in -> width (x n_hidden, GELU) -> n_out; default 6 -> 4 x 128 -> 3."""

    def __init__(self, n_in=6, width=128, n_hidden=4, n_out=3, seed=1):
        import torch
        self.L = _load()
        self.stream = torch.cuda.Stream()
        self.n_in, self.width, self.n_hidden, self.n_out = n_in, width, n_hidden, n_out
        h = ctypes.c_void_p()
        s = self.L.mlp_create(n_in, width, n_hidden, n_out, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if s != 0:
            raise lbm.LbmError(f"mlp_create: {lbm.STATUS.get(s, s)}")
        self._h = h
        self.set_params(self.initial_params(seed))

    def _chk(self, s, what):
        if s != 0:
            m = self.L.mlp_last_error(self._h)
            raise lbm.LbmError(f"{what}: {lbm.STATUS.get(s, s)} ({m.decode() if m else ''})")

    @property
    def n_params(self):
        return self.L.mlp_num_params(self._h)

    def layer_dims(self):
        return [(self.n_in if l == 0 else self.width, self.n_out if l == self.n_hidden else self.width)
                for l in range(self.n_hidden + 1)]

    def initial_params(self, seed):
        """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (seeded)."""
        rng = np.random.default_rng(seed)
        parts = []
        for i, o in self.layer_dims():
            parts.append(rng.uniform(-1.0 / math.sqrt(i), 1.0 / math.sqrt(i), i * o))
            parts.append(np.zeros(o))
        return np.concatenate(parts).astype(np.float32)

    def set_params(self, p):
        p = _f32(p)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.size}")
        self._chk(self.L.mlp_set_params(self._h, p.ctypes.data_as(_fp)), "mlp_set_params")

    def params(self):
        p = np.empty(self.n_params, dtype=np.float32)
        self._chk(self.L.mlp_get_params(self._h, p.ctypes.data_as(_fp)), "mlp_get_params")
        return p

    def forward(self, X):
        X = _f32(X)
        Y = np.empty((X.shape[0], self.n_out), dtype=np.float32)
        self._chk(self.L.mlp_forward(self._h, X.ctypes.data_as(_fp), X.shape[0], Y.ctypes.data_as(_fp)), "mlp_forward")
        return Y

    def loss_grad(self, X, T):
        X, T = _f32(X), _f32(T)
        loss = ctypes.c_double()
        g = np.empty(self.n_params, dtype=np.float32)
        self._chk(self.L.mlp_loss_grad(self._h, X.ctypes.data_as(_fp), T.ctypes.data_as(_fp), X.shape[0],
                                       ctypes.byref(loss), g.ctypes.data_as(_fp)), "mlp_loss_grad")
        return loss.value, g

    def set_data(self, X, T):
        X, T = _f32(X), _f32(T)
        self._chk(self.L.mlp_set_data(self._h, X.ctypes.data_as(_fp), T.ctypes.data_as(_fp), X.shape[0]),
                  "mlp_set_data")

    def train(self, steps, batch=4096, lr=1e-3, seed=7):
        loss = ctypes.c_double()
        self._chk(self.L.mlp_train(self._h, int(steps), int(batch), float(lr), int(seed), ctypes.byref(loss)),
                  "mlp_train")
        return loss.value

    def destroy(self):
        if self._h is not None and self._h.value:
            self.L.mlp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------------------ features

U_SCALE = 0.05


def features(dx, dy, dz, D, tsr, yaw, u_hub):
    """Network inputs for points (dx, dy, dz) relative to a hub (cells)."""
    n = np.broadcast(dx, dy, dz).size
    out = np.empty((n, 6), dtype=np.float32)
    out[:, 0] = np.asarray(dx, dtype=np.float64).reshape(-1) / D
    out[:, 1] = np.asarray(dy, dtype=np.float64).reshape(-1) / D
    out[:, 2] = np.asarray(dz, dtype=np.float64).reshape(-1) / D
    out[:, 3] = (tsr - 6.0) / 3.0
    out[:, 4] = yaw / 0.1
    out[:, 5] = (u_hub - 0.045) / 0.015
    return out


def targets(u_mean, u_hub):
    t = np.asarray(u_mean, dtype=np.float64) / u_hub
    t[:, 0] -= 1.0
    return t.astype(np.float32)


# ------------------------------------------------------------------ data

def wake_grid(hub, D, nx, ny, nz, x_range=(-1.0, 6.0), r_range=1.5, nxs=28, nts=12):
    """Probe points behind a rotor: x/D in x_range, y/D and z/D in
    [-r_range, r_range], clipped to the lattice."""
    xs = np.clip(np.round(hub[0] + np.linspace(x_range[0], x_range[1], nxs) * D), 0, nx - 1).astype(int)
    ys = np.clip(np.round(hub[1] + np.linspace(-r_range, r_range, nts) * D), 0, ny - 1).astype(int)
    zs = np.clip(np.round(hub[2] + np.linspace(-r_range, r_range, nts) * D), 0, nz - 1).astype(int)
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    return X.reshape(-1), Y.reshape(-1), Z.reshape(-1)


def generate_wake_data(n_runs, seed=11, shape=(192, 96, 96), D=24.0, spinup=2000, average=2000, every=20,
                       nu=1e-3):
    """Mean wakes of single-rotor runs with seeded TSR in [4, 8], yaw in
    [0, 10] degrees and U_hub in [0.03, 0.06]: returns (X features, T
    targets, per-run parameters)."""
    from . import inputs as I
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    hub = (2.0 * D, ny / 2.0, nz / 2.0)
    Xs, Ts, runs = [], [], []
    for r in range(n_runs):
        tsr = float(rng.uniform(4.0, 8.0))
        yaw = float(np.radians(rng.uniform(0.0, 10.0)))
        U = float(rng.uniform(0.03, 0.06))
        dom, turb = I.single_turbine_case(nx, ny, nz, diameter=D, hub=hub, elements_per_blade=int(D), tsr=tsr,
                                          u_inf=U, yaw=yaw, nu=nu, seed=int(rng.integers(0, 2 ** 62)))
        lat = lbm.Lattice.create(nx, ny, nz, nu=nu, bc=dom["bc"], seed=dom["seed"])
        lat.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
        lat.add_turbine(**turb)
        lat.step(spinup)
        px, py, pz = wake_grid(hub, D, nx, ny, nz)
        acc = np.zeros((px.size, 3))
        n = 0
        for _ in range(average // every):
            lat.step(every)
            acc += lat.probe(px, py, pz)[1]
            n += 1
        lat.destroy()
        Xs.append(features(px - hub[0], py - hub[1], pz - hub[2], D, tsr, yaw, U))
        Ts.append(targets(acc / n, U))
        runs.append(dict(tsr=tsr, yaw=yaw, U=U))
    return np.concatenate(Xs), np.concatenate(Ts), runs


# ------------------------------------------------------------------ farm warm start

def farm_initial_velocity(net, shape, rotors, inflow_u, stride=4):
    """Initial velocity (3, nz, ny, nx) of a farm: inflow profile inflow_u(z)
    (array of nz values) times (1 - sqrt(sum_t d_t^2)) with d_t = 1 - u_t/U the
    deficit each rotor's surrogate predicts; v and w add the rotors'
    predictions.  Evaluated every `stride` cells and repeated."""
    nx, ny, nz = shape
    xs = np.arange(0, nx, stride) + stride // 2
    ys = np.arange(0, ny, stride) + stride // 2
    zs = np.arange(0, nz, stride) + stride // 2
    xs, ys, zs = np.minimum(xs, nx - 1), np.minimum(ys, ny - 1), np.minimum(zs, nz - 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    d2 = np.zeros(X.shape)
    vw = np.zeros((2,) + X.shape)
    for r in rotors:
        hub, D = r["hub"], r["D"]
        f = features(X - hub[0], Y - hub[1], Z - hub[2], D, r["tsr"], r["yaw"], r["u_hub"])
        p = net.forward(f).reshape(X.shape + (3,)).astype(np.float64)
        # only in the region the network was trained on; outside, no deficit
        inside = ((X - hub[0]) / D >= -1.0) & ((X - hub[0]) / D <= 6.0) & (np.abs(Y - hub[1]) / D <= 1.5) & \
                 (np.abs(Z - hub[2]) / D <= 1.5)
        d = np.where(inside, -p[..., 0], 0.0)
        d2 += np.clip(d, 0.0, 1.0) ** 2
        vw[0] += np.where(inside, p[..., 1], 0.0)
        vw[1] += np.where(inside, p[..., 2], 0.0)
    Uz = np.asarray(inflow_u)[zs][:, None, None]
    coarse = np.stack([Uz * (1.0 - np.sqrt(d2)), Uz * vw[0], Uz * vw[1]])
    full = np.repeat(np.repeat(np.repeat(coarse, stride, axis=1), stride, axis=2), stride, axis=3)
    return full[:, :nz, :ny, :nx]


class WindowMeans:
    """Means of u_x over the cells of a plane, one per window of `window` steps
    (sampled every `every` steps)."""

    def __init__(self, lattice, z, every=50, window=1000):
        self.lat = lattice
        Y, X = np.meshgrid(np.arange(lattice.ny), np.arange(lattice.nx), indexing="ij")
        self.px, self.py = X.reshape(-1), Y.reshape(-1)
        self.pz = np.full(self.px.size, int(z))
        self.every, self.window = every, window
        self.means, self.ends = [], []
        self.step = 0

    def advance(self, steps):
        for _ in range(steps // self.window):
            acc = np.zeros(self.px.size)
            n = 0
            for _ in range(self.window // self.every):
                self.lat.step(self.every)
                acc += self.lat.probe(self.px, self.py, self.pz)[1][:, 0]
                n += 1
            self.step += self.window
            self.means.append(acc / n)
            self.ends.append(self.step)


def converged_reference(wms, from_step):
    """The converged mean (average of the window means after from_step, over
    one run or several) and its noise floor (median relative L2 distance of
    those windows to it)."""
    if isinstance(wms, WindowMeans):
        wms = [wms]
    late = [m for wm in wms for m, e in zip(wm.means, wm.ends) if e > from_step]
    ref = np.mean(late, axis=0)
    noise = float(np.median([np.linalg.norm(m - ref) / np.linalg.norm(ref) for m in late]))
    return ref, noise


def settle_step(wm, ref, tol):
    """First window end at which the window mean is within tol (relative L2) of
    the converged mean; None if it never is."""
    for m, e in zip(wm.means, wm.ends):
        if np.linalg.norm(m - ref) / np.linalg.norm(ref) < tol:
            return e
    return None


def running_mean_changes(wm):
    """Relative L2 change of the running mean of hub-plane u_x over each window:
    with R_k the mean of the first k window means, ||R_k - R_(k-1)|| / ||R_k||
    for k >= 2 (at the window ends 2, 3, ... windows in)."""
    out = []
    acc = np.zeros_like(wm.means[0]) if wm.means else None
    prev = None
    for k, (m, e) in enumerate(zip(wm.means, wm.ends), start=1):
        acc = acc + m
        r = acc / k
        if prev is not None:
            out.append((e, float(np.linalg.norm(r - prev) / np.linalg.norm(r))))
        prev = r
    return out


def running_mean_settle_step(wm, tol=1e-3):
    """First window end at which the running mean of hub-plane u_x changes by
    less than tol (relative L2) over one window: the converged-mean criterion
    of the farm workload.  None if it never does."""
    for e, c in running_mean_changes(wm):
        if c < tol:
            return e
    return None


def window_errors(wm, ref):
    return [float(np.linalg.norm(m - ref) / np.linalg.norm(ref)) for m in wm.means]
