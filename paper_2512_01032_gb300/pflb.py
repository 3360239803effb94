"""Thin ctypes binding of the C ABI in ``include/pflb.h``.

Argument marshalling only: every step of the path runs in the CUDA library.
The names follow the C functions (``pflb_create`` -> ``create`` and so on).
``Lattice`` is a small owner object around the opaque handle.  Streams may
be given as a ``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_P = C.POINTER
_d = _P(C.c_double)

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NAN, ERR_TIMEOUT, ERR_BUDGET, ERR_STATE = range(8)
STORAGE_FP64, STORAGE_FP32, STORAGE_FP16, STORAGE_BF16 = 0, 1, 2, 3
FIELD_PHI, FIELD_RHO, FIELD_P, FIELD_UX, FIELD_UY, FIELD_UZ = range(6)
FIELDS = {"phi": 0, "rho": 1, "P": 2, "ux": 3, "uy": 4, "uz": 5}
KERNEL_FUSED, KERNEL_TWOPASS, KERNEL_FUSED_TMA, KERNEL_PIPE = 0, 1, 2, 3

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NAN",
                5: "ERR_TIMEOUT", 6: "ERR_BUDGET", 7: "ERR_STATE"}


class XBC(C.Structure):
    _fields_ = [("type", C.c_int), ("P", C.c_double), ("u", C.c_double * 3),
                ("phi", C.c_double), ("ramp_steps", C.c_int64)]


XBC_PRESSURE, XBC_VELOCITY = 1, 2


def _xbc(b, ramp_steps=0):
    if b is None:
        return None
    t = {"pressure": XBC_PRESSURE, "velocity": XBC_VELOCITY}.get(b["type"], b["type"])
    u = b.get("u", (0.0, 0.0, 0.0))
    return XBC(int(t), float(b.get("P", 0.0)), (C.c_double * 3)(*u), float(b.get("phi", 0.0)),
               int(ramp_steps))


class DiagRaw(C.Structure):
    _fields_ = [("acc", C.c_double * 32), ("step", C.c_int64), ("err", C.c_int32),
                ("pad", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("storage", C.c_int),
                ("steps_per_tick", C.c_int), ("max_active", C.c_int), ("batched", C.c_int),
                ("max_active_cells", C.c_int64)]


class SolveSpec(C.Structure):
    _fields_ = [("init_shape", C.c_int), ("center", C.c_double * 3), ("R", C.c_double),
                ("normal", C.c_double * 3), ("p_ref", C.c_double), ("length", C.c_double),
                ("dir", C.c_double * 3), ("beta0", C.c_double), ("dbeta", C.c_double),
                ("beta_max", C.c_double), ("ramp_every", C.c_int64), ("max_steps", C.c_int64),
                ("region", C.c_int * 6), ("threshold", C.c_double), ("keep_phi", C.c_int),
                ("drive", C.c_int)]


class SolveResult(C.Structure):
    _fields_ = [("state", C.c_int), ("broke_through", C.c_int), ("beta", C.c_double),
                ("steps", C.c_int64), ("latency_s", C.c_double), ("queue_s", C.c_double),
                ("region_mass", C.c_double), ("mass", C.c_double), ("u_max", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("rejected", C.c_int64), ("active", C.c_int64), ("queued", C.c_int64),
                ("p50_s", C.c_double), ("p99_s", C.c_double), ("mean_s", C.c_double),
                ("max_s", C.c_double), ("makespan_s", C.c_double), ("solves_per_s", C.c_double),
                ("cell_updates", C.c_double), ("bytes_in_use", C.c_size_t),
                ("peak_bytes", C.c_size_t), ("ticks", C.c_int64), ("admit_s", C.c_double),
                ("wait_s", C.c_double), ("retire_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_REJECTED = range(5)


class PflbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("solid", _P(C.c_uint8)), ("wall_normal", _d), ("theta_deg", _d),
                ("solid_frac", _d)]


class Params(C.Structure):
    _fields_ = [
        ("sigma", C.c_double), ("W", C.c_double), ("M", C.c_double), ("rho_H", C.c_double),
        ("rho_L", C.c_double), ("nu_H", C.c_double), ("nu_L", C.c_double),
        ("theta_deg", C.c_double), ("Fex", C.c_double * 3),
        ("gamma", C.c_double), ("phi_M", C.c_double), ("phi_m", C.c_double), ("D", C.c_double),
        ("eps", C.c_double), ("blend", C.c_double), ("band_lo", C.c_double),
        ("band_hi", C.c_double), ("F_tilde", C.c_double), ("F_width", C.c_double),
        ("F_mode", C.c_int), ("mobility_corr", C.c_int), ("free_slip", C.c_int),
        ("storage", C.c_int),
    ]


class Diag(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("mass", C.c_double), ("n_heavy", C.c_double),
        ("p_heavy", C.c_double), ("p_light", C.c_double), ("n_p_heavy", C.c_double),
        ("n_p_light", C.c_double), ("dp", C.c_double), ("u_max", C.c_double),
        ("region_mass", C.c_double), ("cl_count", C.c_double), ("cl_mean", C.c_double * 3),
        ("cl_m2", C.c_double * 3), ("kinetic", C.c_double), ("nonfinite", C.c_double),
        ("front_x", C.c_double), ("rear_x", C.c_double),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, C.Array) else v
        return out


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load ``libpflb.so`` (building it when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path}")
    lib = C.CDLL(path)
    st = C.c_int
    lib.pflb_default_params.argtypes = [_P(Params)]
    lib.pflb_default_params.restype = None
    lib.pflb_create.argtypes = [_P(Geometry), _P(Params), C.c_void_p, _P(C.c_void_p)]
    lib.pflb_create.restype = st
    lib.pflb_init_tanh.argtypes = [C.c_void_p, C.c_int, _d, C.c_double, _d, C.c_double]
    lib.pflb_init_tanh.restype = st
    lib.pflb_init_phi.argtypes = [C.c_void_p, _d, C.c_double]
    lib.pflb_init_phi.restype = st
    lib.pflb_set_force.argtypes = [C.c_void_p, _d]
    lib.pflb_set_force.restype = st
    lib.pflb_set_region.argtypes = [C.c_void_p, _P(C.c_int)]
    lib.pflb_set_region.restype = st
    lib.pflb_set_kernel.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.pflb_set_kernel.restype = st
    lib.pflb_last_diag_async.argtypes = [C.c_void_p, C.c_void_p, _P(C.c_int64)]
    lib.pflb_last_diag_async.restype = st
    lib.pflb_diag_wait.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, _P(Diag)]
    lib.pflb_diag_wait.restype = st
    lib.pflb_set_x_boundaries.argtypes = [C.c_void_p, _P(XBC), _P(XBC)]
    lib.pflb_set_x_boundaries.restype = st
    lib.pflb_selftest_wait_timeout.argtypes = [C.c_void_p, C.c_int64]
    lib.pflb_selftest_wait_timeout.restype = st
    lib.pflb_get_kernel.argtypes = [C.c_void_p, _P(C.c_int)]
    lib.pflb_get_kernel.restype = st
    lib.pflb_tune.argtypes = [C.c_void_p, C.c_int, _P(C.c_int)]
    lib.pflb_tune.restype = st
    lib.pflb_step.argtypes = [C.c_void_p, C.c_int64]
    lib.pflb_step.restype = st
    lib.pflb_step_diag.argtypes = [C.c_void_p, C.c_int64, _P(Diag)]
    lib.pflb_step_diag.restype = st
    lib.pflb_set_diag_every.argtypes = [C.c_void_p, C.c_int]
    lib.pflb_set_diag_every.restype = st
    lib.pflb_last_diag.argtypes = [C.c_void_p, _P(Diag)]
    lib.pflb_last_diag.restype = st
    lib.pflb_read.argtypes = [C.c_void_p, C.c_int, _d]
    lib.pflb_read.restype = st
    lib.pflb_diag.argtypes = [C.c_void_p, _P(Diag)]
    lib.pflb_diag.restype = st
    lib.pflb_get_step.argtypes = [C.c_void_p]
    lib.pflb_get_step.restype = C.c_int64
    lib.pflb_device_bytes.argtypes = [C.c_void_p]
    lib.pflb_device_bytes.restype = C.c_int64
    lib.pflb_estimate_bytes.argtypes = [_P(Geometry), C.c_int]
    lib.pflb_estimate_bytes.restype = C.c_int64
    lib.pflb_save.argtypes = [C.c_void_p, C.c_char_p]
    lib.pflb_save.restype = st
    lib.pflb_load.argtypes = [C.c_void_p, C.c_char_p]
    lib.pflb_load.restype = st
    lib.pflb_destroy.argtypes = [C.c_void_p]
    lib.pflb_destroy.restype = None
    lib.pflb_fields_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                        _P(Params), C.c_void_p, _P(Diag), C.c_void_p]
    lib.pflb_fields_noalloc.restype = st
    lib.pflb_batch_create.argtypes = [_P(C.c_void_p), C.c_int, C.c_void_p, _P(C.c_void_p)]
    lib.pflb_batch_create.restype = st
    lib.pflb_batch_set_launch.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.pflb_batch_set_launch.restype = st
    lib.pflb_batch_tune.argtypes = [C.c_void_p, C.c_int, _P(C.c_int)]
    lib.pflb_batch_tune.restype = st
    lib.pflb_batch_step.argtypes = [C.c_void_p, C.c_int64, C.c_int]
    lib.pflb_batch_step.restype = st
    lib.pflb_batch_destroy.argtypes = [C.c_void_p]
    lib.pflb_batch_destroy.restype = None
    lib.pflb_step_ex.argtypes = [C.c_void_p, C.c_int64, C.c_int]
    lib.pflb_step_ex.restype = st
    lib.pflb_server_create.argtypes = [_P(ServerConfig), C.c_void_p, _P(C.c_void_p)]
    lib.pflb_server_create.restype = st
    lib.pflb_server_submit.argtypes = [C.c_void_p, _P(Geometry), _P(Params), _P(SolveSpec),
                                       _P(C.c_int64)]
    lib.pflb_server_submit.restype = st
    lib.pflb_server_tick.argtypes = [C.c_void_p, _P(C.c_int)]
    lib.pflb_server_tick.restype = st
    lib.pflb_server_poll.argtypes = [C.c_void_p, C.c_int64, _P(SolveResult)]
    lib.pflb_server_poll.restype = st
    lib.pflb_server_fetch_phi.argtypes = [C.c_void_p, C.c_int64, _d, C.c_int64]
    lib.pflb_server_fetch_phi.restype = st
    lib.pflb_server_stats_get.argtypes = [C.c_void_p, _P(ServerStats)]
    lib.pflb_server_stats_get.restype = st
    lib.pflb_server_destroy.argtypes = [C.c_void_p]
    lib.pflb_server_destroy.restype = None
    lib.pflb_last_error.argtypes = []
    lib.pflb_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        msg = load().pflb_last_error().decode(errors="replace")
        raise PflbError(status, msg)


_STORAGE_NAMES = {"fp64": STORAGE_FP64, "fp32": STORAGE_FP32, "fp16": STORAGE_FP16,
                  "bf16": STORAGE_BF16}


def default_params(**kw) -> Params:
    p = Params()
    load().pflb_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "Fex":
            for a in range(3):
                p.Fex[a] = float(v[a])
        elif k == "storage" and isinstance(v, str):
            p.storage = _STORAGE_NAMES[v]
        elif hasattr(p, k):
            setattr(p, k, v)
        else:
            raise KeyError(f"unknown parameter {k}")
    return p


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_geometry(nx, ny, nz, solid=None, wall_normal=None, theta_cells=None, solid_frac=None):
    """Build a ``Geometry`` struct plus the numpy arrays it points into
    (solid_frac: the solid volume fraction of each cell for walls that cut
    fluid cells, or None for voxel walls)."""
    N = int(nx) * int(ny) * int(nz)
    s = np.zeros(N, np.uint8) if solid is None else np.ascontiguousarray(
        np.asarray(solid, np.uint8).reshape(-1))
    if s.size != N:
        raise ValueError("solid mask has the wrong size")
    nw = None if wall_normal is None else _f64(wall_normal).reshape(-1)
    th = None if theta_cells is None else _f64(theta_cells).reshape(-1)
    if nw is not None and nw.size != 3 * N:
        raise ValueError("wall_normal must hold 3 values per cell")
    if th is not None and th.size != N:
        raise ValueError("theta_cells must hold one value per cell")
    fr = None if solid_frac is None else _f64(solid_frac).reshape(-1)
    if fr is not None and fr.size != N:
        raise ValueError("solid_frac must hold one value per cell")
    g = Geometry(int(nx), int(ny), int(nz), s.ctypes.data_as(_P(C.c_uint8)),
                 nw.ctypes.data_as(_d) if nw is not None else None,
                 th.ctypes.data_as(_d) if th is not None else None,
                 fr.ctypes.data_as(_d) if fr is not None else None)
    return g, (s, nw, th, fr)


def fields_noalloc(nx, ny, nz, h_ptr: int, g_ptr: int, params: Params, fields_ptr=None,
                   stream=None, want_diag=True):
    """pflb_fields_noalloc on caller-owned device arrays (raw device
    pointers, e.g. ``tensor.data_ptr()``); returns the diagnostics dict or
    None.  See include/pflb.h for the contract."""
    d = Diag()
    _check(load().pflb_fields_noalloc(int(nx), int(ny), int(nz), C.c_void_p(h_ptr),
                                      C.c_void_p(g_ptr), C.byref(params),
                                      C.c_void_p(fields_ptr) if fields_ptr else None,
                                      C.byref(d) if want_diag else None,
                                      C.c_void_p(_stream_handle(stream))))
    return d.as_dict() if want_diag else None


def estimate_bytes(nx, ny, nz, solid=None, storage=STORAGE_FP32, solid_frac=None) -> int:
    g, keep = make_geometry(nx, ny, nz, solid, solid_frac=solid_frac)
    return int(load().pflb_estimate_bytes(C.byref(g), int(storage)))


class Lattice:
    """Owner of one ``pflb_lattice`` handle."""

    def __init__(self, nx, ny, nz, solid=None, wall_normal=None, theta_cells=None, stream=None,
                 params: Params | None = None, solid_frac=None, **kw):
        lib = load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.params = params if params is not None else default_params(**kw)
        geom, keep = make_geometry(nx, ny, nz, solid, wall_normal, theta_cells, solid_frac)
        self._stream = stream
        h = C.c_void_p()
        _check(lib.pflb_create(C.byref(geom), C.byref(self.params),
                               C.c_void_p(_stream_handle(stream)), C.byref(h)))
        self._h = h
        self._lib = lib

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pflb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- calls
    def init_tanh(self, shape=0, center=(0, 0, 0), R=0.0, normal=None, P0=0.0):
        c = _f64(center)
        n = _f64(normal) if normal is not None else None
        _check(self._lib.pflb_init_tanh(self._h, int(shape), c.ctypes.data_as(_d), float(R),
                                        n.ctypes.data_as(_d) if n is not None else None,
                                        float(P0)))

    def init_phi(self, phi, P0=0.0):
        a = _f64(phi).reshape(-1)
        if a.size != self.N:
            raise ValueError("phi has the wrong size")
        _check(self._lib.pflb_init_phi(self._h, a.ctypes.data_as(_d), float(P0)))

    def set_force(self, F):
        f = _f64(F)
        _check(self._lib.pflb_set_force(self._h, f.ctypes.data_as(_d)))

    def set_region(self, box):
        b = (C.c_int * 6)(*[int(v) for v in box])
        _check(self._lib.pflb_set_region(self._h, b))

    def set_kernel(self, kind=KERNEL_FUSED, bx=0, by=0, lz=0):
        _check(self._lib.pflb_set_kernel(self._h, int(kind), int(bx), int(by), int(lz)))

    def last_diag_async(self, raw_ptr: int) -> int:
        """Queue a copy of the last diagnostics into the DiagRaw at host
        address raw_ptr (page-locked for an asynchronous copy); returns a
        ticket for diag_wait."""
        t = C.c_int64()
        _check(self._lib.pflb_last_diag_async(self._h, C.c_void_p(raw_ptr), C.byref(t)))
        return t.value

    def diag_wait(self, ticket: int, raw_ptr: int, allow_nan=False) -> dict:
        d = Diag()
        s = self._lib.pflb_diag_wait(self._h, int(ticket), C.c_void_p(raw_ptr), C.byref(d))
        if not (allow_nan and s == ERR_NAN):
            _check(s)
        return d.as_dict()

    def set_x_boundaries(self, lo=None, hi=None, ramp_steps=0):
        """Open x boundaries: lo / hi dicts with type ("pressure" or
        "velocity"), P, u (3), phi; None for both restores periodic x.
        ramp_steps > 0 reaches the values linearly over that many steps."""
        a, b = _xbc(lo, ramp_steps), _xbc(hi, ramp_steps)
        _check(self._lib.pflb_set_x_boundaries(self._h, C.byref(a) if a else None,
                                               C.byref(b) if b else None))

    def selftest_wait_timeout(self, polls=1000):
        """Queue the bounded-wait self-test (the next synchronising call
        reports ERR_TIMEOUT and poisons this lattice)."""
        _check(self._lib.pflb_selftest_wait_timeout(self._h, int(polls)))

    def get_kernel(self) -> dict:
        out = (C.c_int * 4)()
        _check(self._lib.pflb_get_kernel(self._h, out))
        return dict(kind=out[0], bx=out[1], by=out[2], lz=out[3])

    def tune(self, trial_steps=50) -> int:
        """Pick the fastest planes per block for the kernel in effect by
        timing real steps (the lattice advances); returns the chosen lz."""
        lz = C.c_int(0)
        _check(self._lib.pflb_tune(self._h, int(trial_steps), C.byref(lz)))
        return lz.value

    def step(self, n=1):
        _check(self._lib.pflb_step(self._h, int(n)))

    def step_diag(self, n=1) -> dict:
        d = Diag()
        _check(self._lib.pflb_step_diag(self._h, int(n), C.byref(d)))
        return d.as_dict()

    def set_diag_every(self, k: int):
        _check(self._lib.pflb_set_diag_every(self._h, int(k)))

    def last_diag(self, allow_nan=False) -> dict:
        d = Diag()
        s = self._lib.pflb_last_diag(self._h, C.byref(d))
        if s != OK and not (allow_nan and s == ERR_NAN):
            _check(s)
        return d.as_dict()

    def read(self, field) -> np.ndarray:
        f = FIELDS[field] if isinstance(field, str) else int(field)
        out = np.empty(self.N, np.float64)
        _check(self._lib.pflb_read(self._h, f, out.ctypes.data_as(_d)))
        return out

    def read_all(self) -> dict:
        return {k: self.read(k) for k in FIELDS}

    def diag(self, allow_nan=False) -> dict:
        d = Diag()
        s = self._lib.pflb_diag(self._h, C.byref(d))
        if s != OK and not (allow_nan and s == ERR_NAN):
            _check(s)
        return d.as_dict()

    @property
    def t(self) -> int:
        return int(self._lib.pflb_get_step(self._h))

    def device_bytes(self) -> int:
        return int(self._lib.pflb_device_bytes(self._h))

    def save(self, path):
        _check(self._lib.pflb_save(self._h, os.fsencode(path)))

    def load(self, path):
        _check(self._lib.pflb_load(self._h, os.fsencode(path)))


class Batch:
    """Many lattices advanced together by one persistent kernel (the lattices
    stay owned by the caller and must outlive the batch)."""

    def __init__(self, lattices, stream=None):
        self._lib = load()
        self.lattices = list(lattices)
        arr = (C.c_void_p * len(self.lattices))(*[L.handle.value for L in self.lattices])
        h = C.c_void_p()
        _check(self._lib.pflb_batch_create(arr, len(self.lattices),
                                           C.c_void_p(_stream_handle(stream)), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pflb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_launch(self, bx=0, by=0, lz=0, blocks_per_sm=0):
        _check(self._lib.pflb_batch_set_launch(self._h, int(bx), int(by), int(lz),
                                               int(blocks_per_sm)))

    def tune(self, trial_steps=4) -> tuple:
        best = (C.c_int * 4)()
        _check(self._lib.pflb_batch_tune(self._h, int(trial_steps), best))
        return tuple(best)

    def step(self, n=1, diag_last=False):
        _check(self._lib.pflb_batch_step(self._h, int(n), 1 if diag_last else 0))


class Server:
    """Request server with continuous batching (``pflb_server``).

    ``submit`` takes a geometry (solid mask, optional normals and angles),
    model parameters and a solve spec (dict with the SolveSpec fields);
    ``tick`` advances the resident requests; ``poll`` / ``stats`` report."""

    def __init__(self, hbm_budget_bytes=16 << 30, storage="fp32", steps_per_tick=250,
                 max_active=0, batched=True, max_active_cells=0, stream=None):
        self._lib = load()
        self.storage = _STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
        cfg = ServerConfig(int(hbm_budget_bytes), self.storage, int(steps_per_tick),
                           int(max_active), 1 if batched else 0, int(max_active_cells))
        h = C.c_void_p()
        _check(self._lib.pflb_server_create(C.byref(cfg), C.c_void_p(_stream_handle(stream)),
                                            C.byref(h)))
        self._h = h
        self._dims = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pflb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, nx, ny, nz, spec: dict, solid=None, wall_normal=None, theta_cells=None,
               **params) -> int:
        params.pop("storage", None)  # every request runs at the server's storage
        p = default_params(storage=self.storage, **params)
        g, keep = make_geometry(nx, ny, nz, solid, wall_normal, theta_cells)
        sp = SolveSpec()
        for k, v in spec.items():
            f = getattr(sp, k)
            if isinstance(f, C.Array):
                for i, x in enumerate(v):
                    f[i] = x
            else:
                setattr(sp, k, v)
        t = C.c_int64()
        _check(self._lib.pflb_server_submit(self._h, C.byref(g), C.byref(p), C.byref(sp),
                                            C.byref(t)))
        self._dims[t.value] = int(nx) * int(ny) * int(nz)
        return t.value

    def tick(self) -> int:
        n = C.c_int()
        _check(self._lib.pflb_server_tick(self._h, C.byref(n)))
        return n.value

    def poll(self, ticket) -> dict:
        r = SolveResult()
        _check(self._lib.pflb_server_poll(self._h, int(ticket), C.byref(r)))
        return r.as_dict()

    def fetch_phi(self, ticket) -> np.ndarray:
        n = self._dims[int(ticket)]
        out = np.empty(n, np.float64)
        _check(self._lib.pflb_server_fetch_phi(self._h, int(ticket), out.ctypes.data_as(_d), n))
        return out

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.pflb_server_stats_get(self._h, C.byref(st)))
        return st.as_dict()
