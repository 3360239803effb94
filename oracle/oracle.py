"""ctypes front end of the FP64 oracle in ``pflb_oracle.c``.

Test infrastructure only (see the package docstring).  The C file is compiled
with gcc on first use into ``oracle/_build/``; no CUDA code is involved.
The tanh initial profile of Eq. 12 (``tanh_phi``) is written here, for the
oracle's own use, independently of the library's ``init_tanh``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pflb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math) and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class OrcParams(C.Structure):
    _fields_ = [
        ("sigma", C.c_double), ("W", C.c_double), ("M", C.c_double),
        ("rho_H", C.c_double), ("rho_L", C.c_double),
        ("nu_H", C.c_double), ("nu_L", C.c_double),
        ("theta_deg", C.c_double),
        ("Fex", C.c_double * 3),
        ("gamma", C.c_double), ("phi_M", C.c_double), ("phi_m", C.c_double),
        ("D", C.c_double), ("eps", C.c_double),
        ("blend", C.c_double),
        ("band_lo", C.c_double), ("band_hi", C.c_double),
        ("F_tilde", C.c_double), ("F_width", C.c_double),
        ("F_mode", C.c_int), ("mobility_corr", C.c_int), ("free_slip", C.c_int),
        ("nthreads", C.c_int),
    ]


_P = C.POINTER
_d = _P(C.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle())
        lib.orc_create.restype = C.c_void_p
        lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, _P(C.c_uint8), _d, _d, _P(OrcParams)]
        lib.orc_destroy.argtypes = [C.c_void_p]
        lib.orc_init_phi.argtypes = [C.c_void_p, _d, C.c_double]
        lib.orc_step.argtypes = [C.c_void_p, C.c_int64]
        lib.orc_macros.argtypes = [C.c_void_p] + [_d] * 6
        lib.orc_get_step.restype = C.c_int64
        lib.orc_get_step.argtypes = [C.c_void_p]
        for n in ("orc_get_h", "orc_get_g", "orc_set_h", "orc_set_g", "orc_get_ghost",
                  "orc_set_ghost", "orc_set_phi_field", "orc_get_normals"):
            getattr(lib, n).argtypes = [C.c_void_p, _d]
        lib.orc_update_ghosts_only.argtypes = [C.c_void_p]
        lib.orc_set_solid_fraction.argtypes = [C.c_void_p, _d, _d]
        lib.orc_set_solid_fraction.restype = C.c_int
        lib.orc_set_nthreads.argtypes = [C.c_void_p, C.c_int]
        lib.orc_set_force.argtypes = [C.c_void_p, _d]
        lib.orc_set_x_boundaries.argtypes = [C.c_void_p, C.c_int, _d, C.c_int, _d, C.c_int64]
        lib.orc_set_x_boundaries.restype = C.c_int
        lib.orc_lattice_tables.argtypes = [_P(C.c_int), _P(C.c_int), _P(C.c_int), _d, _P(C.c_int)]
        lib.orc_max_threads.restype = C.c_int
        lib.orc_gamma.argtypes = [_d, _d]
        lib.orc_cd_stencil.argtypes = [_d, _d, _d]
        lib.orc_chem_pot.restype = C.c_double
        lib.orc_chem_pot.argtypes = [_P(OrcParams), C.c_double, C.c_double]
        lib.orc_delta_theta.restype = C.c_double
        lib.orc_delta_theta.argtypes = [_P(OrcParams), C.c_double, _d, C.c_double]
        lib.orc_h_eq.argtypes = [_P(OrcParams), C.c_double, _d, _d, C.c_double, _d]
        lib.orc_tau_mix.restype = C.c_double
        lib.orc_tau_mix.argtypes = [_P(OrcParams), C.c_double]
        lib.orc_macros_cell.argtypes = [_P(OrcParams), _d, C.c_double, _d, C.c_double,
                                        _d, _d, _d, _d]
        lib.orc_force_and_eq.argtypes = [_P(OrcParams), C.c_double, C.c_double, _d, C.c_double,
                                         _d, _d, _d]
        lib.orc_filtered_collide.argtypes = [_d, _d, _d, C.c_double, _d, _d]
        lib.orc_ghost_values.argtypes = [_P(OrcParams), C.c_double, _d, C.c_double, C.c_double,
                                         _d, C.c_uint32, _d]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_d)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


DEFAULTS = dict(
    sigma=0.01, W=4.0, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=0.1, nu_L=0.1, theta_deg=90.0,
    Fex=(0.0, 0.0, 0.0), gamma=-22.5, phi_M=0.8, phi_m=0.2, D=1e-4, eps=1e-10, blend=0.95,
    band_lo=0.5, band_hi=0.95, F_tilde=0.1, F_width=0.001, F_mode=0, mobility_corr=1,
    free_slip=0, nthreads=1,
)


def make_params(**kw) -> OrcParams:
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError(f"unknown oracle parameters: {sorted(unknown)}")
    d.update(kw)
    p = OrcParams()
    for k, v in d.items():
        if k == "Fex":
            for a in range(3):
                p.Fex[a] = float(v[a])
        else:
            setattr(p, k, v)
    return p


def lattice_tables():
    lib = _load()
    cx = (C.c_int * 19)(); cy = (C.c_int * 19)(); cz = (C.c_int * 19)()
    w = (C.c_double * 19)(); opp = (C.c_int * 19)()
    lib.orc_lattice_tables(cx, cy, cz, w, opp)
    c = np.stack([np.array(cx[:]), np.array(cy[:]), np.array(cz[:])], axis=1)
    return c, np.array(w[:]), np.array(opp[:])


# ----------------------------------------------------------- per-cell hooks

def gamma_vec(u):
    lib = _load(); u = _f64(u); out = np.zeros(19)
    lib.orc_gamma(_ptr(u), _ptr(out)); return out


def cd_stencil(val):
    lib = _load(); val = _f64(val); grad = np.zeros(3); lap = np.zeros(1)
    lib.orc_cd_stencil(_ptr(val), _ptr(grad), _ptr(lap)); return grad, float(lap[0])


def chem_pot(params: OrcParams, phi, lap):
    return _load().orc_chem_pot(C.byref(params), float(phi), float(lap))


def delta_theta(params: OrcParams, phi, grad, lap):
    g = _f64(grad)
    return _load().orc_delta_theta(C.byref(params), float(phi), _ptr(g), float(lap))


def h_eq(params: OrcParams, phi, u, grad, lap):
    lib = _load(); u = _f64(u); g = _f64(grad); out = np.zeros(19)
    lib.orc_h_eq(C.byref(params), float(phi), _ptr(u), _ptr(g), float(lap), _ptr(out)); return out


def tau_mix(params: OrcParams, phi):
    return _load().orc_tau_mix(C.byref(params), float(phi))


def macros_cell(params: OrcParams, g, phi, grad, lap):
    lib = _load(); g = _f64(g); gr = _f64(grad)
    rho = np.zeros(1); P = np.zeros(1); u = np.zeros(3); mu = np.zeros(1)
    lib.orc_macros_cell(C.byref(params), _ptr(g), float(phi), _ptr(gr), float(lap),
                        _ptr(rho), _ptr(P), _ptr(u), _ptr(mu))
    return float(rho[0]), float(P[0]), u, float(mu[0])


def force_and_eq(params: OrcParams, rho, P, u, mu, grad):
    lib = _load(); u = _f64(u); gr = _f64(grad); K = np.zeros(19); E = np.zeros(19)
    lib.orc_force_and_eq(C.byref(params), float(rho), float(P), _ptr(u), float(mu), _ptr(gr),
                         _ptr(K), _ptr(E))
    return K, E


def filtered_collide(g, K, E, tau):
    lib = _load(); g = _f64(g); K = _f64(K); E = _f64(E); gs = np.zeros(19); Pi = np.zeros(9)
    lib.orc_filtered_collide(_ptr(g), _ptr(K), _ptr(E), float(tau), _ptr(gs), _ptr(Pi))
    return gs, Pi.reshape(3, 3)


def ghost_values(params: OrcParams, phi_smpl, nw, theta_deg, grad, solid_links: int):
    lib = _load(); nw = _f64(nw); gr = _f64(grad); out = np.full(19, np.nan)
    th = np.deg2rad(theta_deg)
    lib.orc_ghost_values(C.byref(params), float(phi_smpl), _ptr(nw), float(np.cos(th)),
                         float(np.sin(th)), _ptr(gr), C.c_uint32(solid_links), _ptr(out))
    return out


def cell_collide(params: OrcParams, g, phi, grad, lap):
    """Macros, K, E and the filtered post-collision g for one cell."""
    rho, P, u, mu = macros_cell(params, g, phi, grad, lap)
    K, E = force_and_eq(params, rho, P, u, mu, grad)
    gs, Pi = filtered_collide(g, K, E, tau_mix(params, phi))
    return dict(rho=rho, P=P, u=u, mu=mu, K=K, E=E, gstar=gs, Pi=Pi)


# ----------------------------------------------------------- initial field

def tanh_phi(shape, nxyz, center, radius, W, normal=(1.0, 0.0, 0.0)):
    """Initial order parameter from the steady tanh profile of Eq. 12.

    shape 0: sphere, phi = (1 + tanh(2 (R - r)/W))/2 with r the minimum-image
    distance from ``center`` (cell centres at integer coordinates).
    shape 1: half space, phi = (1 + tanh(2 d/W))/2 with d = (c - x) . normal.
    shape 2: slab of half width R about ``center`` along ``normal``.
    """
    nx, ny, nz = nxyz
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = []
    for coord, n, c in ((x, nx, center[0]), (y, ny, center[1]), (z, nz, center[2])):
        dd = coord - c
        dd = dd - n * np.round(dd / n)
        d.append(dd)
    if shape == 0:
        arg = radius - np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    else:
        nn = np.asarray(normal, dtype=np.float64)
        nn = nn / np.linalg.norm(nn)
        s = d[0] * nn[0] + d[1] * nn[1] + d[2] * nn[2]
        arg = -s if shape == 1 else radius - np.abs(s)
    return (0.5 * (1.0 + np.tanh(2.0 * arg / W))).reshape(-1)


# ----------------------------------------------------------- lattice object

class OracleLattice:
    """One periodic lattice advanced by the FP64 oracle."""

    def __init__(self, nx, ny, nz, solid=None, wall_normal=None, theta_cells=None, nthreads=1,
                 solid_frac=None, **params):
        """solid_frac: optional solid volume fraction per cell (reading R23:
        walls that cut fluid cells); fluid cells in [0, 1)."""
        lib = _load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.params = make_params(nthreads=nthreads, **params)
        solid = np.zeros(self.N, np.uint8) if solid is None else np.ascontiguousarray(
            np.asarray(solid, dtype=np.uint8).reshape(-1))
        if solid.size != self.N:
            raise ValueError("solid mask has the wrong size")
        self.solid = solid
        nw = None if wall_normal is None else _f64(wall_normal).reshape(-1)
        th = None if theta_cells is None else _f64(theta_cells).reshape(-1)
        if nw is not None and nw.size != 3 * self.N:
            raise ValueError("wall_normal must hold 3 values per cell")
        if th is not None and th.size != self.N:
            raise ValueError("theta_cells must hold one angle per cell")
        self._keep = (solid, nw, th)
        self._h = lib.orc_create(self.nx, self.ny, self.nz, solid.ctypes.data_as(_P(C.c_uint8)),
                                 _ptr(nw) if nw is not None else None,
                                 _ptr(th) if th is not None else None, C.byref(self.params))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self._lib = lib
        if solid_frac is not None:
            fr = _f64(solid_frac).reshape(-1)
            if fr.size != self.N:
                raise ValueError("solid_frac must hold one value per cell")
            self._keep = self._keep + (fr,)
            if lib.orc_set_solid_fraction(self._h, _ptr(fr),
                                          _ptr(nw) if nw is not None else None) != 0:
                raise ValueError("solid_frac of a fluid cell outside [0, 1)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def init_phi(self, phi0, P0: float = 0.0):
        a = _f64(phi0).reshape(-1)
        self._lib.orc_init_phi(self._h, _ptr(a), float(P0))

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    @property
    def t(self) -> int:
        return int(self._lib.orc_get_step(self._h))

    def set_nthreads(self, n: int):
        self._lib.orc_set_nthreads(self._h, int(n))

    def set_force(self, F):
        f = _f64(F)
        self._lib.orc_set_force(self._h, _ptr(f))

    def set_x_boundaries(self, lo=None, hi=None, ramp_steps=0):
        """Open x boundaries (reading R22): lo / hi are dicts with type
        ("pressure" or "velocity"), P, u (3) and phi; None for both restores
        periodic x.  ramp_steps > 0 reaches the given values linearly from
        those in effect (the rest state when the boundaries were off)."""
        kinds = {None: 0, "pressure": 1, "velocity": 2}

        def pack(b):
            if b is None:
                return 0, np.zeros(5)
            u = b.get("u", (0.0, 0.0, 0.0))
            return kinds[b["type"]], _f64([b.get("P", 0.0), u[0], u[1], u[2], b.get("phi", 0.0)])

        tl, vl = pack(lo)
        th, vh = pack(hi)
        if self._lib.orc_set_x_boundaries(self._h, tl, _ptr(vl), th, _ptr(vh),
                                          int(ramp_steps)) != 0:
            raise ValueError("bad open-boundary request")

    def macros(self):
        out = [np.zeros(self.N) for _ in range(6)]
        self._lib.orc_macros(self._h, *[_ptr(a) for a in out])
        phi, rho, P, ux, uy, uz = out
        return dict(phi=phi, rho=rho, P=P, ux=ux, uy=uy, uz=uz)

    def _get(self, name, width):
        a = np.zeros(self.N * width)
        getattr(self._lib, name)(self._h, _ptr(a))
        return a.reshape(self.N, width)

    def populations(self):
        return self._get("orc_get_h", 19), self._get("orc_get_g", 19)

    def set_populations(self, h, g):
        h = _f64(h).reshape(-1); g = _f64(g).reshape(-1)
        self._lib.orc_set_h(self._h, _ptr(h)); self._lib.orc_set_g(self._h, _ptr(g))

    def ghosts(self):
        return self._get("orc_get_ghost", 19)

    def set_ghosts(self, gh):
        a = _f64(gh).reshape(-1)
        self._lib.orc_set_ghost(self._h, _ptr(a))

    def set_phi_field(self, phi):
        a = _f64(phi).reshape(-1)
        self._lib.orc_set_phi_field(self._h, _ptr(a))

    def update_ghosts_only(self):
        self._lib.orc_update_ghosts_only(self._h)

    def normals(self):
        return self._get("orc_get_normals", 3)
