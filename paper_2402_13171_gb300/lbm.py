"""Thin ctypes binding of the C ABI in include/lbm_gb300.h.

Argument marshalling only: every step of the solver runs in the CUDA library
(liblbm_gb300.so).  PyTorch provides device memory (its caching allocator,
passed to the library as dev_alloc/dev_free) and the CUDA stream.  There is no
fallback: if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm_gb300.so")

LBM_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error", 4: "non-finite state",
          5: "device wait timed out", 6: "invalid state", 7: "unsupported combination"}
COLL = {"cumulant": 0, "srt_smag": 1}
STORE = {"fp32": 0, "bf16": 1, "fp16": 2}
BC = {"periodic": 0, "inout": 1, "noslip": 2, "freeslip": 3}
STORE_BYTES = {"fp32": 4, "bf16": 2, "fp16": 2}

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class LbmConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("nu", ctypes.c_double), ("smag_c", ctypes.c_double),
        ("storage", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("body_force", ctypes.c_double * 3),
        ("seed", ctypes.c_ulonglong),
        ("diag_every", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("tile_z", ctypes.c_int),
        ("staged", ctypes.c_int),
        ("inplace", ctypes.c_int),
    ]


class LbmInflow(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u_ref", ctypes.c_double * 3), ("z0", ctypes.c_double),
                ("z_ref", ctypes.c_double), ("noise_rel", ctypes.c_double)]


class AlmTurbineDesc(ctypes.Structure):
    _fields_ = [
        ("hub", ctypes.c_double * 3), ("radius", ctypes.c_double),
        ("n_blades", ctypes.c_int), ("n_elements", ctypes.c_int),
        ("epsilon", ctypes.c_double), ("omega", ctypes.c_double),
        ("yaw", ctypes.c_double), ("pitch", ctypes.c_double), ("theta0", ctypes.c_double),
        ("chord_root", ctypes.c_double), ("chord_tip", ctypes.c_double),
        ("twist", _dp), ("n_polar", ctypes.c_int),
        ("alpha", _dp), ("cl", _dp), ("cd", _dp),
        ("regularisation", ctypes.c_int),
        ("tip_loss", ctypes.c_int),
    ]


REGULARISATION = {"gauss": 0, "roma": 1}


class LbmError(RuntimeError):
    pass


def _require(ok, what):
    """Argument check of the binding (kept under python -O, unlike assert)."""
    if not ok:
        raise ValueError(what)


_lib = None


def load():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LbmError(f"CUDA library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    ctx_pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "lbm_create": [ctypes.POINTER(LbmConfig), ctx_pp],
        "lbm_batch_create": [ctypes.c_int, ctypes.POINTER(LbmConfig), ctx_pp],
        "lbm_set_inflow": [ctypes.c_void_p, ctypes.POINTER(LbmInflow)],
        "lbm_init_fields": [ctypes.c_void_p, _dp, _dp, _fp],
        "alm_add_turbine": [ctypes.c_void_p, ctypes.POINTER(AlmTurbineDesc), ctypes.POINTER(ctypes.c_int)],
        "lbm_step": [ctypes.c_void_p, ctypes.c_int],
        "lbm_sync": [ctypes.c_void_p],
        "lbm_get_moments": [ctypes.c_void_p, _dp, _dp],
        "lbm_get_pdfs": [ctypes.c_void_p, _dp],
        "lbm_set_pdfs": [ctypes.c_void_p, _dp],
        "alm_get_loads": [ctypes.c_void_p, ctypes.c_int, _dp, _dp, _fp, _fp],
        "alm_get_loads_async": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
        "alm_set_loads_sink": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
        "lbm_get_diagnostics": [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_longlong)],
        "lbm_get_step": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)],
        "lbm_set_step": [ctypes.c_void_p, ctypes.c_longlong],
        "lbm_set_profiling": [ctypes.c_void_p, ctypes.c_int],
        "lbm_get_kernel_time": [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_longlong)],
        "lbm_get_traffic_model": [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_longlong)],
        "lbm_get_launches_per_step": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)],
        "lbm_set_tile": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "lbm_probe": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, _dp, _dp],
        "lbm_autotune": [ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_double)],
        "lbm_get_tile": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "lbm_get_state_size": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)],
        "lbm_get_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
        "lbm_set_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
        "lbm_set_wait_limit": [ctypes.c_void_p, ctypes.c_longlong],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.lbm_last_error.argtypes = [ctypes.c_void_p]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_status_string.argtypes = [ctypes.c_int]
    L.lbm_status_string.restype = ctypes.c_char_p
    L.lbm_destroy.argtypes = [ctypes.c_void_p]
    L.lbm_destroy.restype = None
    _lib = L
    return L


def _p(a, ptr=_dp):
    return None if a is None else a.ctypes.data_as(ptr)


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, on the context's stream."""

    def __init__(self, stream):
        import torch
        self.torch = torch
        self.stream = stream
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.stream.device, self.stream)
        except Exception:
            return None

    def _free(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)


def make_config(nx, ny, nz, collision="cumulant", nu=0.01, smag_c=0.0, storage="fp32",
                bc=("periodic", "periodic", "periodic"), body_force=(0.0, 0.0, 0.0), seed=0, diag_every=0,
                tile=(0, 0), stream_ptr=None, allocator=None, inplace=False) -> LbmConfig:
    c = LbmConfig()
    c.nx, c.ny, c.nz = int(nx), int(ny), int(nz)
    c.collision = COLL[collision] if isinstance(collision, str) else int(collision)
    c.nu = float(nu)
    c.smag_c = float(smag_c)
    c.storage = STORE[storage] if isinstance(storage, str) else int(storage)
    for a in range(3):
        c.bc[a] = BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
        c.body_force[a] = float(body_force[a])
    c.seed = int(seed) & ((1 << 64) - 1)
    c.diag_every = int(diag_every)
    c.cuda_stream = stream_ptr
    if allocator is not None:
        c.dev_alloc = allocator.alloc_cb
        c.dev_free = allocator.free_cb
    c.tile_x, c.tile_y = int(tile[0]), int(tile[1])
    c.tile_z = int(tile[2]) if len(tile) > 2 else 0
    c.staged = int(tile[3]) if len(tile) > 3 else 0
    c.inplace = int(bool(inplace))
    return c


class Lattice:
    """One lattice handle.  Use ``Lattice.create`` or ``batch_create``."""

    def __init__(self, handle, shape, keep, storage):
        self._h = ctypes.c_void_p(handle)
        self.nx, self.ny, self.nz = shape
        self.N = self.nx * self.ny * self.nz
        self._keep = keep  # allocator callbacks / stream shared by a batch
        self.storage = storage
        self.turbines = []
        self._sink = None

    # -------------------------------------------------------------- creation
    @staticmethod
    def _stream_and_alloc(device=0):
        import torch
        stream = torch.cuda.Stream(device=device)
        return stream, _TorchAllocator(stream)

    @classmethod
    def create(cls, nx, ny, nz, device=0, **kw):
        L = load()
        stream, alloc = cls._stream_and_alloc(device)
        cfg = make_config(nx, ny, nz, stream_ptr=stream.cuda_stream, allocator=alloc, **kw)
        h = ctypes.c_void_p()
        _check_status(L.lbm_create(ctypes.byref(cfg), ctypes.byref(h)), None, "lbm_create")
        return cls(h.value, (nx, ny, nz), {"stream": stream, "alloc": alloc, "cfg": cfg}, kw.get("storage", "fp32"))

    def _call(self, name, *args):
        L = load()
        s = getattr(L, name)(self._h, *args)
        _check_status(s, self._h, name)
        return s

    @property
    def stream(self):
        return self._keep["stream"]

    # -------------------------------------------------------------- ABI calls
    def set_inflow(self, u_ref=(0.05, 0.0, 0.0), kind=0, z0=0.1, z_ref=1.0, noise_rel=0.0):
        inf = LbmInflow()
        inf.kind = int(kind)
        for a in range(3):
            inf.u_ref[a] = float(u_ref[a])
        inf.z0 = float(z0)
        inf.z_ref = float(z_ref)
        inf.noise_rel = float(noise_rel)
        self._call("lbm_set_inflow", ctypes.byref(inf))

    def init_fields(self, rho=None, u=None, fneq=None):
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        v = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        g = None if fneq is None else np.ascontiguousarray(fneq, dtype=np.float32).reshape(-1)
        if r is not None:
            _require(r.size == self.N, "rho needs nx*ny*nz values")
        if v is not None:
            _require(v.size == 3 * self.N, "u needs 3*nx*ny*nz values")
        if g is not None:
            _require(g.size == 27 * self.N, "fneq needs 27*nx*ny*nz values")
        self._call("lbm_init_fields", _p(r), _p(v), _p(g, _fp))

    def add_turbine(self, hub, radius, n_blades, n_elements, epsilon, omega, alpha, cl, cd, yaw=0.0, pitch=0.0,
                    theta0=0.0, chord_root=1.0, chord_tip=1.0, twist=None, kernel="gauss", tip_loss=False):
        """Add a rotor; `kernel` is the force regularisation, "gauss" (width
        epsilon) or "roma" (Roma et al.'s three-point delta, epsilon unused);
        `tip_loss` applies Glauert's tip-loss factor to the element forces."""
        arrs = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in
                dict(alpha=alpha, cl=cl, cd=cd).items()}
        tw = None if twist is None else np.ascontiguousarray(twist, dtype=np.float64)
        d = AlmTurbineDesc()
        for a in range(3):
            d.hub[a] = float(hub[a])
        d.radius = float(radius)
        d.n_blades = int(n_blades)
        d.n_elements = int(n_elements)
        d.epsilon = float(epsilon)
        d.omega = float(omega)
        d.yaw, d.pitch, d.theta0 = float(yaw), float(pitch), float(theta0)
        d.chord_root, d.chord_tip = float(chord_root), float(chord_tip)
        d.twist = _p(tw)
        d.n_polar = arrs["alpha"].size
        d.alpha, d.cl, d.cd = _p(arrs["alpha"]), _p(arrs["cl"]), _p(arrs["cd"])
        d.regularisation = REGULARISATION[kernel] if isinstance(kernel, str) else int(kernel)
        d.tip_loss = int(tip_loss)
        tid = ctypes.c_int()
        self._call("alm_add_turbine", ctypes.byref(d), ctypes.byref(tid))
        self.turbines.append(int(n_blades) * int(n_elements))
        self._sink = None  # the library clears the loads sink when a rotor is added
        return tid.value

    def step(self, n=1):
        self._call("lbm_step", int(n))

    def sync(self):
        self._call("lbm_sync")

    def moments(self, rho=None, u=None):
        """rho (nz, ny, nx) and u (3, nz, ny, nx) as float64, into new arrays or
        into the caller's (C-contiguous float64 arrays of N and 3N values, for
        example views of page-locked memory, which the device copies into
        directly)."""
        if rho is None:
            rho = np.empty((self.nz, self.ny, self.nx))
        if u is None:
            u = np.empty((3, self.nz, self.ny, self.nx))
        for a, n in ((rho, self.N), (u, 3 * self.N)):
            _require(a.dtype == np.float64 and a.flags.c_contiguous and a.size == n,
                     "moment outputs must be C-contiguous float64 arrays of N and 3N values")
        self._call("lbm_get_moments", _p(rho), _p(u))
        return rho, u

    def probe(self, x, y, z):
        """rho (n) and u (n, 3) at cells (x, y, z) (integer arrays of equal length)."""
        x, y, z = (np.asarray(v, dtype=np.int64).reshape(-1) for v in (x, y, z))
        cells = np.ascontiguousarray((z * self.ny + y) * self.nx + x, dtype=np.int64)
        rho = np.empty(cells.size)
        u = np.empty((cells.size, 3))
        self._call("lbm_probe", cells.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), int(cells.size), _p(rho),
                   _p(u))
        return rho, u

    def pdfs(self):
        f = np.empty((27, self.nz, self.ny, self.nx))
        self._call("lbm_get_pdfs", _p(f))
        return f

    def set_pdfs(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64)
        _require(a.size == 27 * self.N, "PDFs need 27*nx*ny*nz values")
        self._call("lbm_set_pdfs", _p(a))

    def state(self):
        """Checkpoint blob (numpy uint8 array) for a bitwise resume with set_state."""
        n = ctypes.c_size_t()
        self._call("lbm_get_state_size", ctypes.byref(n))
        buf = np.empty(n.value, dtype=np.uint8)
        self._call("lbm_get_state", ctypes.c_void_p(buf.ctypes.data), n)
        return buf

    def set_state(self, buf):
        a = np.ascontiguousarray(buf, dtype=np.uint8)
        self._call("lbm_set_state", ctypes.c_void_p(a.ctypes.data), ctypes.c_size_t(a.size))

    def set_wait_limit(self, cycles):
        """Bound of the staged step's copy-barrier waits (SM clock cycles)."""
        self._call("lbm_set_wait_limit", ctypes.c_longlong(int(cycles)))

    def loads(self, tid=0, elements=False):
        th = ctypes.c_double()
        tq = ctypes.c_double()
        ne = self.turbines[tid]
        ef = np.empty((ne, 3), dtype=np.float32) if elements else None
        ep = np.empty((ne, 3), dtype=np.float32) if elements else None
        self._call("alm_get_loads", int(tid), ctypes.byref(th), ctypes.byref(tq), _p(ef, _fp), _p(ep, _fp))
        if elements:
            return th.value, tq.value, ef, ep
        return th.value, tq.value

    def loads_async(self, out, tid=0):
        """Enqueue the copy of the last enqueued step's (thrust, torque) into
        `out`, a page-locked float64 torch tensor of 2 elements, on the
        lattice's stream; read it after an event recorded behind it."""
        _require(out.dtype == self._torch().float64 and out.numel() == 2 and out.is_pinned(),
                 "out must be a page-locked float64 tensor of 2 elements")
        self._call("alm_get_loads_async", int(tid), ctypes.c_void_p(out.data_ptr()))

    def set_loads_sink(self, ring):
        """Have the device write each step's (thrust, torque) of every rotor
        into `ring`, a page-locked float64 torch tensor of shape
        (ring_len, n_turb, 2): step s lands in ring[s % ring_len] once step
        s - 1 has finished on the stream.  None clears the sink."""
        if ring is None:
            self._call("alm_set_loads_sink", None, 0)
            self._sink = None
            return
        _require(ring.dtype == self._torch().float64 and ring.is_pinned() and ring.is_contiguous(),
                 "the ring must be a contiguous page-locked float64 tensor")
        _require(ring.dim() == 3 and ring.shape[1] == len(self.turbines) and ring.shape[2] == 2,
                 "the ring must have shape (ring_len, rotors, 2)")
        self._call("alm_set_loads_sink", ctypes.c_void_p(ring.data_ptr()), int(ring.shape[0]))
        self._sink = ring  # keep it alive while the device writes to it

    @staticmethod
    def _torch():
        import torch
        return torch

    def diagnostics(self):
        out = np.zeros(4)
        at = ctypes.c_longlong()
        self._call("lbm_get_diagnostics", _p(out), ctypes.byref(at))
        return out, at.value

    def step_count(self):
        n = ctypes.c_longlong()
        self._call("lbm_get_step", ctypes.byref(n))
        return n.value

    def set_step(self, n):
        self._call("lbm_set_step", ctypes.c_longlong(int(n)))

    def set_profiling(self, on=True):
        self._call("lbm_set_profiling", int(bool(on)))

    def kernel_time(self):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        self._call("lbm_get_kernel_time", ctypes.byref(ms), ctypes.byref(n))
        return ms.value, n.value

    def set_tile(self, tx, ty, tz=1, staged=0):
        self._call("lbm_set_tile", int(tx), int(ty), int(tz), int(staged))

    def autotune(self, steps=20, cache=None):
        out = (ctypes.c_int * 4)()
        ms = ctypes.c_double()
        self._call("lbm_autotune", int(steps), None if cache is None else str(cache).encode(), out, ctypes.byref(ms))
        return tuple(out), ms.value

    def tile(self):
        """(tile_x, tile_y, tile_z, staged)."""
        v = [ctypes.c_int() for _ in range(4)]
        self._call("lbm_get_tile", *[ctypes.byref(a) for a in v])
        return tuple(a.value for a in v)

    def traffic_model(self):
        b = ctypes.c_double()
        n = ctypes.c_longlong()
        self._call("lbm_get_traffic_model", ctypes.byref(b), ctypes.byref(n))
        return b.value, n.value

    def launches_per_step(self):
        n = ctypes.c_int()
        self._call("lbm_get_launches_per_step", ctypes.byref(n))
        return n.value

    def destroy(self):
        if self._h is not None and self._h.value:
            load().lbm_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def batch_create(cfgs, device=0):
    """cfgs: list of dicts of make_config keyword arguments (nx, ny, nz, ...).
    Returns one Lattice per instance; stepping any steps all."""
    L = load()
    stream, alloc = Lattice._stream_and_alloc(device)
    arr = (LbmConfig * len(cfgs))()
    for i, kw in enumerate(cfgs):
        kw = dict(kw)
        nx, ny, nz = kw.pop("nx"), kw.pop("ny"), kw.pop("nz")
        arr[i] = make_config(nx, ny, nz, stream_ptr=stream.cuda_stream, allocator=alloc, **kw)
    hs = (ctypes.c_void_p * len(cfgs))()
    _check_status(L.lbm_batch_create(len(cfgs), arr, hs), None, "lbm_batch_create")
    keep = {"stream": stream, "alloc": alloc, "cfg": arr}
    return [Lattice(hs[i], (cfgs[i]["nx"], cfgs[i]["ny"], cfgs[i]["nz"]), keep,
                    cfgs[i].get("storage", "fp32")) for i in range(len(cfgs))]


def _check_status(s, handle, what):
    if s != LBM_OK:
        msg = ""
        if handle is not None:
            m = load().lbm_last_error(handle)
            msg = m.decode() if m else ""
        raise LbmError(f"{what}: {STATUS.get(s, s)} ({msg})")


def header_functions():
    """Names of the functions declared in include/lbm_gb300.h."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "lbm_gb300.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:lbm_status|const char\*|void)\s+\**(\w+)\s*\(", text, re.M)))
