"""Seeded synthetic inputs: voxelised geometry, wall normals and workload
recipes for the capillary-flow cases.

This module holds no arithmetic of the lattice Boltzmann method.  It builds
the data both the oracle and the CUDA library take as input: a solid mask
(uint8, x fastest), unit wall normals pointing into the fluid (from the
analytic shapes' signed distance), per-cell input contact angles, and the
parameter sets of each workload.  The initial order parameter is not built
here: each side computes its own tanh profile.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


# ------------------------------------------------------------------ shapes

@dataclasses.dataclass
class Plane:
    """Solid half space {x : (x - point) . normal < 0}; normal points into fluid."""
    point: tuple
    normal: tuple

    def sdf(self, X, Y, Z):
        n = np.asarray(self.normal, float); n = n / np.linalg.norm(n)
        p = self.point
        return (X - p[0]) * n[0] + (Y - p[1]) * n[1] + (Z - p[2]) * n[2]

    def grad(self, X, Y, Z):
        n = np.asarray(self.normal, float); n = n / np.linalg.norm(n)
        return [np.full_like(X, n[0], dtype=float), np.full_like(X, n[1], dtype=float),
                np.full_like(X, n[2], dtype=float)]


@dataclasses.dataclass
class Sphere:
    """Solid ball of radius R (cell centres at integer coordinates)."""
    center: tuple
    R: float

    def sdf(self, X, Y, Z):
        c = self.center
        return np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - self.R

    def grad(self, X, Y, Z):
        c = self.center
        d = np.stack([X - c[0], Y - c[1], Z - c[2]]).astype(float)
        r = np.sqrt((d ** 2).sum(0))
        r = np.where(r == 0, 1.0, r)
        return [d[0] / r, d[1] / r, d[2] / r]


@dataclasses.dataclass
class Box:
    """Solid axis-aligned box [lo, hi) in cell coordinates."""
    lo: tuple
    hi: tuple

    def sdf(self, X, Y, Z):
        # distance-like: positive outside, negative inside (per-axis max)
        ds = []
        for A, l, h in ((X, self.lo[0], self.hi[0]), (Y, self.lo[1], self.hi[1]),
                        (Z, self.lo[2], self.hi[2])):
            ds.append(np.maximum(l - 0.5 - A, A - (h - 0.5)))
        return np.maximum(np.maximum(ds[0], ds[1]), ds[2])

    def grad(self, X, Y, Z):
        ds = []
        for A, l, h in ((X, self.lo[0], self.hi[0]), (Y, self.lo[1], self.hi[1]),
                        (Z, self.lo[2], self.hi[2])):
            ds.append((l - 0.5 - A, A - (h - 0.5)))
        # normal along the axis with the largest positive distance
        cand = []
        for a in range(3):
            lo_d, hi_d = ds[a]
            cand.append((np.maximum(lo_d, hi_d), np.where(hi_d >= lo_d, 1.0, -1.0)))
        best = np.argmax(np.stack([c[0] for c in cand]), axis=0)
        g = [np.zeros_like(X, dtype=float) for _ in range(3)]
        for a in range(3):
            g[a] = np.where(best == a, cand[a][1], 0.0)
        return g


_OFFS = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
         if (abs(dx) + abs(dy) + abs(dz)) in (1, 2)]


class Geometry:
    """Voxelised solid geometry on a periodic nx*ny*nz box (x fastest)."""

    def __init__(self, nx, ny, nz, shapes=(), theta_deg=90.0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.shapes = list(shapes)
        Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        self._XYZ = (X.astype(float), Y.astype(float), Z.astype(float))
        solid = np.zeros((nz, ny, nx), bool)
        for s in self.shapes:
            solid |= s.sdf(*self._XYZ) < 0
        self.solid3 = solid
        self.theta3 = np.full((nz, ny, nx), float(theta_deg))
        # solid volume fraction of fluid cells that a wall cuts (0: voxel walls)
        self.frac3 = np.zeros((nz, ny, nx))

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    @property
    def solid(self) -> np.ndarray:
        return self.solid3.astype(np.uint8).reshape(-1)

    def wall_nodes3(self) -> np.ndarray:
        """Fluid cells with at least one solid or cut D3Q19 neighbour."""
        s = self.solid3
        sc = s | (self.frac3 > 0)
        w = np.zeros_like(s)
        for dx, dy, dz in _OFFS:
            w |= np.roll(sc, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        return w & ~s

    def solid_frac(self):
        """Solid volume fraction per cell (x fastest), or None for voxel walls."""
        if not (self.frac3 > 0).any():
            return None
        return np.where(self.solid3, 1.0, self.frac3).reshape(-1)

    def normals(self) -> np.ndarray:
        """Unit wall normals (into the fluid) at wall nodes, zero elsewhere.

        Each wall node takes the normal of the shape whose surface is nearest
        (smallest signed distance), from that shape's analytic gradient."""
        X, Y, Z = self._XYZ
        wn = self.wall_nodes3()
        n = np.zeros(self.solid3.shape + (3,))
        if not self.shapes:
            return n.reshape(-1)
        sd = np.stack([s.sdf(X, Y, Z) for s in self.shapes])
        best = np.argmin(sd, axis=0)
        for k, s in enumerate(self.shapes):
            g = s.grad(X, Y, Z)
            sel = wn & (best == k)
            for a in range(3):
                n[..., a] = np.where(sel, g[a], n[..., a])
        nn = np.linalg.norm(n, axis=-1, keepdims=True)
        n = np.where(nn > 0, n / np.where(nn > 0, nn, 1.0), 0.0)
        return n.reshape(-1)

    def theta(self) -> np.ndarray:
        return self.theta3.reshape(-1).copy()

    def set_theta_near(self, shape_index: int, theta_deg: float):
        """Give wall nodes nearest to one shape their own contact angle."""
        X, Y, Z = self._XYZ
        sd = np.stack([s.sdf(X, Y, Z) for s in self.shapes])
        best = np.argmin(sd, axis=0)
        self.theta3 = np.where(best == shape_index, float(theta_deg), self.theta3)


# -------------------------------------------------------------- workloads

def static_droplet_params():
    """Periodic static 3-D droplet: 32^3, R=8, W=4 at the box centre; density
    ratio 1000, sigma=0.01, tau_H=tau_L=0.8, M=0.02, plain model."""
    return dict(sigma=0.01, W=4.0, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=0.1, nu_L=0.1,
                F_mode=0, mobility_corr=1, free_slip=0, blend=0.0)


def static_droplet(n=32, R=8.0):
    """Droplet at the box centre ((n-1)/2 in cell coordinates 0..n-1, i.e.
    between lattice sites, so that no cell sits on a mirror plane where
    grad phi vanishes exactly)."""
    g = Geometry(n, n, n)
    c = (n - 1) / 2.0
    return g, static_droplet_params(), dict(shape=0, center=(c, c, c), R=R)


def sessile_sphere_params(theta_deg=90.0):
    """Droplet on a curved wall: density ratio 1000, sigma=0.005, W=4,
    tau=0.8, M=0.02, optimised model (tanh F, free-slip band, blend 0.95)."""
    return dict(sigma=0.005, W=4.0, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=0.1, nu_L=0.1,
                theta_deg=theta_deg, F_mode=1, mobility_corr=1, free_slip=1, blend=0.95)


def sessile_sphere(n=128, theta_deg=90.0):
    """n^3 box, solid sphere radius 30*(n/128) centred on the bottom plane,
    solid planes at z=0 and z=n-1, droplet of radius 20*(n/128) tangent to the
    sphere's top (all lengths scale with n)."""
    s = n / 128.0
    c = (n - 1) / 2.0  # box centre, between lattice sites
    shapes = [Sphere((c, c, 0.0), 30.0 * s), Plane((0, 0, 0.5), (0, 0, 1)),
              Plane((0, 0, n - 1.5), (0, 0, -1))]
    g = Geometry(n, n, n, shapes, theta_deg=theta_deg)
    g.set_theta_near(1, 90.0)
    g.set_theta_near(2, 90.0)
    drop = dict(shape=0, center=(c, c, 30.0 * s + 20.0 * s), R=20.0 * s)
    return g, sessile_sphere_params(theta_deg), drop


def slit_params():
    """Capillary filling: theta=45, density ratio 1000, viscosity ratio 50
    (nu_H = 1/60, nu_L = 1/3), sigma=0.01, M=0.1666, W=4 (W=2.5 with these
    relaxation times is unstable at the free interface)."""
    return dict(sigma=0.01, W=4.0, M=0.1666, rho_H=1.0, rho_L=1e-3, nu_H=1.0 / 60.0,
                nu_L=1.0 / 3.0, theta_deg=45.0, F_mode=1, mobility_corr=1, free_slip=1,
                blend=0.95)


def slit(nx=1024, ny=64, nz=4, reservoir=128):
    """Two-plate slit: walls at y=0 and y=ny-1 for reservoir <= x < nx-reservoir,
    periodic box; liquid slab in the left reservoir."""
    shapes = [Box((reservoir, 0, -10 ** 6), (nx - reservoir, 1, 10 ** 6)),
              Box((reservoir, ny - 1, -10 ** 6), (nx - reservoir, ny, 10 ** 6))]
    g = Geometry(nx, ny, nz, shapes, theta_deg=45.0)
    drop = dict(shape=2, center=(reservoir / 2.0 - 0.5, 0, 0), R=reservoir / 2.0,
                normal=(1, 0, 0))
    return g, slit_params(), drop


def channel_batch_specs(count=64, seed=2512010320):
    """Uneven droplet-in-square-channel lattices: Ny=Nz~U{32..96},
    Nx~U{96..384}, drop radius ~U[0.3,0.45]*Ny at x=Nx/4, theta~U[40,140],
    driving speed ~U[1e-4,1e-3] (applied as a body force)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        ny = int(rng.integers(32, 97))
        nx = int(rng.integers(96, 385))
        rr = float(rng.uniform(0.3, 0.45)) * ny
        th = float(rng.uniform(40.0, 140.0))
        u = float(rng.uniform(1e-4, 1e-3))
        out.append(dict(nx=nx, ny=ny, nz=ny, R=rr, theta=th, u_in=u))
    return out


def static_slug(theta_deg, H=32, length=64, nx=192, nz=4):
    """Liquid slug at rest between two flat plates (the gap is H fluid cells:
    solid rows y = 0 and y = H + 1, periodic in x and z): liquid for
    |x - nx/2 + 1/2| < length/2 with flat initial menisci; theta on both
    plates, density ratio 1000, sigma = 0.01, W = 4, tau = 0.8, M = 0.02,
    optimised model (tanh F, free-slip band, ghost blend 0.95: the flat
    initial menisci are far from the wetting angle, and without the blend
    the jump at 160 degrees drives the light phase unstable within 40 steps)."""
    ny = H + 2
    shapes = [Plane((0, 0.5, 0), (0, 1, 0)), Plane((0, ny - 1.5, 0), (0, -1, 0))]
    g = Geometry(nx, ny, nz, shapes, theta_deg=theta_deg)
    p = dict(sigma=0.01, W=4.0, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=0.1, nu_L=0.1,
             theta_deg=theta_deg, F_mode=1, mobility_corr=1, free_slip=1, blend=0.95)
    init = dict(shape=2, center=(nx / 2.0 - 0.5, 0.0, 0.0), R=length / 2.0, normal=(1.0, 0.0, 0.0))
    return g, p, init


def offset_slug(theta_deg, delta, H=32, length=64, nx=192, nz=4):
    """The static slug between flat plates with both walls moved into the
    channel by delta in [0, 1) (Sec. IV A: the lattice-aligned walls at 0
    and H become delta and H - delta): solid rows y = 0 and y = H + 1 as in
    static_slug, and the rows y = 1 and y = H cut by the walls with solid
    fraction delta (the walls at y = 0.5 + delta and H + 0.5 - delta).  The
    gap between the walls is H - 2 delta.  Voxels count as solid only when
    the wall covers them whole, so the cut rows stay fluid cells."""
    g, p, init = static_slug(theta_deg, H=H, length=length, nx=nx, nz=nz)
    if not 0.0 <= delta < 1.0:
        raise ValueError("delta must lie in [0, 1)")
    g.frac3[:, 1, :] = delta
    g.frac3[:, H, :] = delta
    g.shapes = [Plane((0, 0.5 + delta, 0), (0, 1, 0)),
                Plane((0, H + 0.5 - delta, 0), (0, -1, 0))]
    return g, p, init


def dynamic_slug(U=2e-3, H=32, nx=384, length=64, theta_deg=133.0, nz=4):
    """Liquid slug driven along a slit (plates H cells apart, periodic in z)
    by a gas velocity inlet U at x = 0 against a pressure outlet at x = nx-1:
    the 2-D analogue of the paper's Sec. IV B channel (hydrophobic walls,
    theta 133 degrees).  Density ratio 1000, dynamic viscosity ratio 50
    (nu_H = 1/60, nu_L = 1/3), sigma = 0.01, W = 4, M = 0.1666, optimised
    model.  The slug starts at rest with flat menisci for 64 <= x < 64 +
    length."""
    ny = H + 2
    shapes = [Plane((0, 0.5, 0), (0, 1, 0)), Plane((0, ny - 1.5, 0), (0, -1, 0))]
    g = Geometry(nx, ny, nz, shapes, theta_deg=theta_deg)
    p = dict(sigma=0.01, W=4.0, M=0.1666, rho_H=1.0, rho_L=1e-3, nu_H=1.0 / 60.0,
             nu_L=1.0 / 3.0, theta_deg=theta_deg, F_mode=1, mobility_corr=1, free_slip=1,
             blend=0.95)
    init = dict(shape=2, center=(64 + length / 2.0 - 0.5, 0.0, 0.0), R=length / 2.0,
                normal=(1.0, 0.0, 0.0))
    inlet = dict(type="velocity", u=(U, 0.0, 0.0), phi=0.0)
    outlet = dict(type="pressure", P=0.0)
    return g, p, init, inlet, outlet


def channel_lattice(spec: dict):
    """(geometry, params, init) of one channel_batch_specs entry: square duct
    along x, droplet at x = Nx/4 on the axis, carrier driven by a uniform body
    force giving the mean laminar speed u_in of a square duct of side a
    (mean u = f a^2 / (28.45 rho nu) for a force density f)."""
    nx, ny, nz = spec["nx"], spec["ny"], spec["nz"]
    g = square_channel(nx, ny, nz, spec["theta"])
    p = sessile_sphere_params(spec["theta"])
    a = ny - 2.0
    f = 28.45 * p["rho_L"] * p["nu_L"] * spec["u_in"] / (a * a)
    p = dict(p, Fex=(f, 0.0, 0.0))
    init = dict(shape=0, center=(nx / 4.0, (ny - 1) / 2.0, (nz - 1) / 2.0), R=spec["R"])
    return g, p, init


def square_channel(nx, ny, nz, theta_deg):
    """Square duct along x: walls on the four sides (y, z = 0 and n-1)."""
    shapes = [Plane((0, 0.5, 0), (0, 1, 0)), Plane((0, ny - 1.5, 0), (0, -1, 0)),
              Plane((0, 0, 0.5), (0, 0, 1)), Plane((0, 0, nz - 1.5), (0, 0, -1))]
    return Geometry(nx, ny, nz, shapes, theta_deg=theta_deg)


def constriction_channel(w, ratio, theta_deg):
    """Square channel of width w and length 4w with a central square
    constriction of side ratio*w and length w."""
    nx, ny, nz = 4 * w, w + 2, w + 2
    d = max(2, int(round(ratio * w)))
    lo = (ny - d) // 2
    x0, x1 = int(1.5 * w), int(2.5 * w)
    shapes = [Plane((0, 0.5, 0), (0, 1, 0)), Plane((0, ny - 1.5, 0), (0, -1, 0)),
              Plane((0, 0, 0.5), (0, 0, 1)), Plane((0, 0, nz - 1.5), (0, 0, -1)),
              Box((x0, 0, 0), (x1, lo, nz)), Box((x0, lo + d, 0), (x1, ny, nz)),
              Box((x0, 0, 0), (x1, ny, lo)), Box((x0, 0, lo + d), (x1, ny, nz))]
    return Geometry(nx, ny, nz, shapes, theta_deg=theta_deg), d


def constriction_params(theta_deg):
    """Slug through a constriction: density ratio 1000, dynamic viscosity
    ratio 50 (nu_H = 1/60, nu_L = 1/3), sigma = 0.01, W = 4, M = 0.1666,
    optimised model."""
    return dict(sigma=0.01, W=4.0, M=0.1666, rho_H=1.0, rho_L=1e-3, nu_H=1.0 / 60.0,
                nu_L=1.0 / 3.0, theta_deg=theta_deg, F_mode=1, mobility_corr=1, free_slip=1,
                blend=0.95)


def critical_pressure(sigma, theta_deg, d, H):
    """Capillary entry pressure of a square constriction of side d in a square
    duct of side H (3-D square-duct analogue of the paper's 2-D estimate):
    4 sigma |cos theta| (1/d - 1/H)."""
    return 4.0 * sigma * abs(math.cos(math.radians(theta_deg))) * (1.0 / d - 1.0 / H)


def constriction_request(req: dict, ramp_every=2000, max_steps=26000):
    """Geometry, parameters, initial slug and breakthrough test of one
    serving_trace entry.  The slug (liquid, phi = 1) fills the duct for
    0.25 w <= x < 1.25 w, upstream of the constriction [1.5 w, 2.5 w).  The
    pressure ramp is a body force F_x with F_x L = beta P_crit (L = 4 w, the
    periodic length), beta = 0.7, 0.75, ... raised every ramp_every steps up
    to 1.3.  Breakthrough: liquid volume beyond the constriction exit + W
    (region 2.5 w + W <= x < 3.75 w) above half a constriction cross-section."""
    w = req["w"]
    g, d = constriction_channel(w, req["ratio"], req["theta"])
    p = constriction_params(req["theta"])
    pc = critical_pressure(p["sigma"], req["theta"], d, w)
    init = dict(shape=2, center=(0.75 * w - 0.5, 0.0, 0.0), R=0.5 * w, normal=(1.0, 0.0, 0.0))
    x_lo = int(math.ceil(2.5 * w + p["W"]))
    region = (x_lo, int(3.75 * w), 0, g.ny, 0, g.nz)  # x0, x1, y0, y1, z0, z1
    return dict(geometry=g, params=p, init=init, d=d, p_crit=pc, length=float(g.nx),
                beta0=0.7, dbeta=0.05, beta_max=1.3, ramp_every=ramp_every,
                max_steps=max_steps, region=region, threshold=0.5 * d * d)


def constriction_spec(r: dict, keep_phi=False, drive="force") -> dict:
    """The pflb_solve_spec fields of a constriction_request; drive "force"
    applies the ramp pressure as a body force over the periodic length,
    "pressure" as the pressure difference across open x boundaries."""
    i = r["init"]
    return dict(init_shape=i["shape"], center=i["center"], R=i["R"], normal=i["normal"],
                p_ref=r["p_crit"], length=r["length"], dir=(1.0, 0.0, 0.0), beta0=r["beta0"],
                dbeta=r["dbeta"], beta_max=r["beta_max"], ramp_every=r["ramp_every"],
                max_steps=r["max_steps"], region=r["region"], threshold=r["threshold"],
                keep_phi=1 if keep_phi else 0, drive={"force": 0, "pressure": 1}[drive])


def serving_trace(count=200, rate=20.0, seed=2512010321):
    """Poisson arrivals of critical-pressure solves (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for k in range(count):
        out.append(dict(t_arrival=float(t[k]), w=int(rng.integers(48, 97)),
                        ratio=float(rng.uniform(0.3, 0.7)),
                        theta=float(rng.uniform(90.0, 150.0))))
    return out


def cap_angle_from_volume_height(V: float, h: float) -> float:
    """Contact angle (deg) of a spherical cap with volume V and height h
    (V = pi h^2 (3r - h)/3, cos theta = 1 - h/r)."""
    r = (3.0 * V / (math.pi * h * h) + h) / 3.0
    return math.degrees(math.acos(max(-1.0, min(1.0, 1.0 - h / r))))


def fit_circle(points: np.ndarray):
    """Least-squares circle through 2-D points: returns (cx, cy, r)."""
    P = np.asarray(points, float)
    A = np.c_[2 * P[:, 0], 2 * P[:, 1], np.ones(len(P))]
    b = (P ** 2).sum(1)
    s = np.linalg.lstsq(A, b, rcond=None)[0]
    return s[0], s[1], math.sqrt(s[2] + s[0] ** 2 + s[1] ** 2)


def contour_points(phi2: np.ndarray, level=0.5):
    """phi=level crossings of a 2-D slice phi2[row=z, col=x] along rows and
    columns (linear interpolation), as (x, z) points."""
    pts = []
    nz, nx = phi2.shape
    a = phi2 - level
    for z in range(nz):
        r = a[z]
        idx = np.where(r[:-1] * r[1:] < 0)[0]
        for x in idx:
            pts.append((x + r[x] / (r[x] - r[x + 1]), z))
    for x in range(nx):
        c = a[:, x]
        idx = np.where(c[:-1] * c[1:] < 0)[0]
        for z in idx:
            pts.append((x, z + c[z] / (c[z] - c[z + 1])))
    return np.array(pts, float).reshape(-1, 2)
