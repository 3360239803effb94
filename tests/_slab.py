"""A z-slab decomposition of the oracle's time step, for testing the
single-lattice multi-GPU design on CPU ranks (test infrastructure).

Each slab owns the planes z0 <= z < z1 of an nx * ny * nz lattice: their
populations, wall ghosts, wall normals and angles.  The solid mask is
geometry and is replicated.  One step runs the oracle's sub-steps in its
order (reading R3): phi = sum h; wall ghosts from the previous ghosts (R11)
and the blend (R12); the Eq. 13 stencil; macros, the h collision (Eqs. 1-4)
and the filtered g collision (Eqs. 5-11); push streaming with halfway
bounce-back (R13).  Every per-cell quantity comes from the oracle's own C
routines, so a slab does exactly the arithmetic of the undecomposed step.

What crosses a slab face each step, and nothing else:
  - before the ghosts and stencils: the slab's first and last plane of phi
    (the neighbours' halo planes), nx * ny values per face;
  - after the collision: the populations that stream out through the face,
    5 directions per population set (those with c_z = -1 or +1), nx * ny
    values each per face.
So each face cell costs 1 + 2 * 5 = 11 values per step (44 B at FP32).
The free-slip band (R14) can send a population across a face too: an edge
link into a wall whose tangent has a z component is reflected onto the
neighbour x + (0, 0, c_z), possibly in the next slab.  It lands in a slot
(that cell, a direction with c_z = +-1) whose ordinary source is the solid
cell, so it travels in the same 5-direction message, in a place ordinary
streaming leaves empty: the exchange does not grow.  Open x boundaries
(R22) are slab-local as well: a boundary cell's state comes from the
adjacent cell in x, in the same z plane, and its phi_b reaches the
neighbouring slab's stencils through the phi plane, which is formed after
the boundary states.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from oracle.oracle import make_params

Q = 19
CV, _W, OPP = O.lattice_tables()
DOWN = [i for i in range(Q) if CV[i, 2] == -1]
UP = [i for i in range(Q) if CV[i, 2] == 1]


class Slab:
    def __init__(self, dims, z0, z1, solid3, normals, theta, kw, h, g, ghost, xbc=None):
        self.nx, self.ny, self.nz = dims
        self.z0, self.z1 = z0, z1
        self.kw = kw
        self.p = make_params(**kw)
        self.tau_phi = kw["M"] / (1.0 / 3.0) + 0.5
        self.solid3 = solid3.astype(bool)
        plane = self.nx * self.ny
        own = slice(z0 * plane, z1 * plane)
        self.h = h[own].copy()
        self.g = g[own].copy()
        self.ghost = ghost[own].copy()
        self.nw = normals[own].copy()
        self.theta = theta[own].copy()
        self.phi = np.zeros((z1 - z0, self.ny, self.nx))
        self.halo_lo = self.halo_hi = None
        self.values_sent = 0
        self.reflected_across = 0
        self.xbc = xbc  # None, or the (x = 0, x = nx - 1) boundary specs
        self.bstate = {}

    # -- indexing
    def owns(self, z):
        return self.z0 <= z < self.z1

    def idx(self, z, y, x):
        return ((z - self.z0) * self.ny + y) * self.nx + x

    def phi_at(self, z, y, x):
        if self.owns(z):
            return self.phi[z - self.z0, y, x]
        if z == (self.z0 - 1) % self.nz:
            return self.halo_lo[y, x]
        assert z == self.z1 % self.nz, z
        return self.halo_hi[y, x]

    def cells(self):
        for z in range(self.z0, self.z1):
            for y in range(self.ny):
                for x in range(self.nx):
                    yield z, y, x

    def nbr(self, z, y, x, i):
        return ((z + CV[i, 2]) % self.nz, (y + CV[i, 1]) % self.ny, (x + CV[i, 0]) % self.nx)

    # -- the step
    def compute_phi(self):
        for z, y, x in self.cells():
            if self.solid3[z, y, x]:
                self.phi[z - self.z0, y, x] = 0.0
                continue
            s = 0.0
            for v in self.h[self.idx(z, y, x)]:
                s += float(v)
            self.phi[z - self.z0, y, x] = s

    def boundary_side(self, z, y, x):
        if self.xbc is None or self.solid3[z, y, x]:
            return -1
        return 0 if x == 0 else (1 if x == self.nx - 1 else -1)

    def boundary_states(self):
        """Reading R22 for the owned planes: each boundary cell's (phi_b, P_b,
        u_b) from the given values and the adjacent interior cell's pre-step
        bulk moments; phi of the boundary cell becomes phi_b."""
        if self.xbc is None:
            return
        kw, T = self.kw, 1.0 / 3.0
        F = kw.get("Fex", (0.0, 0.0, 0.0))
        for z in range(self.z0, self.z1):
            for y in range(self.ny):
                for side, xb, xa in ((0, 0, 1), (1, self.nx - 1, self.nx - 2)):
                    spec = self.xbc[side]
                    phia, Pa, ua = 0.0, 0.0, [0.0, 0.0, 0.0]
                    if not self.solid3[z, y, xa]:
                        g = self.g[self.idx(z, y, xa)]
                        s0, m = 0.0, [0.0, 0.0, 0.0]
                        for i in range(Q):
                            s0 += g[i]
                            for a in range(3):
                                m[a] += CV[i, a] * g[i]
                        phia = self.phi[z - self.z0, y, xa]
                        rho = kw["rho_L"] + phia * (kw["rho_H"] - kw["rho_L"])
                        ua = [(m[a] + 0.5 * F[a]) / rho for a in range(3)]
                        Pa = T * s0
                    if spec["type"] == "pressure":
                        st = (phia, spec["P"], ua)
                    else:
                        st = (spec["phi"], Pa, list(spec["u"]))
                    if not self.solid3[z, y, xb]:
                        self.phi[z - self.z0, y, xb] = st[0]
                    self.bstate[(z, y, side)] = st

    def face_planes(self):
        """(first plane, last plane) of phi: sent to the slab below / above."""
        self.values_sent += 2 * self.nx * self.ny
        return self.phi[0].copy(), self.phi[-1].copy()

    def stencil(self, z, y, x, ghost):
        c = self.idx(z, y, x)
        val = [self.phi[z - self.z0, y, x]]
        mask = 0
        for i in range(1, Q):
            t = self.nbr(z, y, x, i)
            if self.solid3[t]:
                val.append(ghost[c, i])
                mask |= 1 << i
            else:
                val.append(self.phi_at(*t))
        grad, lap = O.cd_stencil(val)
        return grad, lap, mask

    def update_ghosts(self):
        old = self.ghost.copy()
        b = self.kw.get("blend", 0.95)
        for z, y, x in self.cells():
            if self.solid3[z, y, x] or self.boundary_side(z, y, x) >= 0:
                continue
            c = self.idx(z, y, x)
            grad, _, mask = self.stencil(z, y, x, old)
            if not mask:
                continue
            fresh = O.ghost_values(self.p, self.phi[z - self.z0, y, x], self.nw[c],
                                   self.theta[c], grad, mask)
            for i in range(1, Q):
                if mask >> i & 1:
                    self.ghost[c, i] = b * old[c, i] + (1.0 - b) * fresh[i]

    def collide_and_stream(self):
        """Collide every owned fluid cell and push its populations; returns
        the populations leaving through the lower and upper faces, as
        [direction][y][x] arrays for h and g (NaN where nothing is sent)."""
        nx, ny = self.nx, self.ny
        self.h2 = np.zeros_like(self.h)
        self.g2 = np.zeros_like(self.g)
        out = {k: np.full((5, ny, nx), np.nan) for k in ("lo_h", "lo_g", "hi_h", "hi_g")}
        for z, y, x in self.cells():
            if self.solid3[z, y, x]:
                continue
            c = self.idx(z, y, x)
            f = self.phi[z - self.z0, y, x]
            side = self.boundary_side(z, y, x)
            if side >= 0:
                phi_b, P_b, u_b = self.bstate[(z, y, side)]
                G = O.gamma_vec(u_b)
                rho_b = self.kw["rho_L"] + phi_b * (self.kw["rho_H"] - self.kw["rho_L"])
                hs = phi_b * G
                gs = _W * P_b / (1.0 / 3.0) + rho_b * (G - _W)
            else:
                grad, lap, _ = self.stencil(z, y, x, self.ghost)
                rho, P, u, mu = O.macros_cell(self.p, self.g[c], f, grad, lap)
                heq = O.h_eq(self.p, f, u, grad, lap)
                hs = self.h[c] - (self.h[c] - heq) / self.tau_phi
                K, E = O.force_and_eq(self.p, rho, P, u, mu, grad)
                gs, _ = O.filtered_collide(self.g[c], K, E, O.tau_mix(self.p, f))
            for i in range(Q):
                t = self.nbr(z, y, x, i)
                if self.solid3[t]:
                    self.h2[c, OPP[i]] = hs[i]
                    sp = (self.specular(z, y, x, i, f)
                          if self.kw.get("free_slip") and side < 0 else None)
                    if sp is None:
                        self.g2[c, OPP[i]] = gs[i]
                    else:
                        self.put_g(sp[0], sp[1], gs[i], out)
                elif self.owns(t[0]):
                    self.h2[self.idx(*t), i] = hs[i]
                    self.g2[self.idx(*t), i] = gs[i]
                elif t[0] == (self.z0 - 1) % self.nz:
                    j = DOWN.index(i)
                    out["lo_h"][j, t[1], t[2]] = hs[i]
                    out["lo_g"][j, t[1], t[2]] = gs[i]
                else:
                    j = UP.index(i)
                    out["hi_h"][j, t[1], t[2]] = hs[i]
                    out["hi_g"][j, t[1], t[2]] = gs[i]
        self.values_sent += 4 * 5 * nx * ny
        return out

    def specular(self, z, y, x, i, f):
        """Reading R14: the edge link i of wall node (z, y, x) into a solid
        cell, whose step along one of its two axes is solid and along the
        other fluid, is reflected across the solid axis onto the tangential
        neighbour when phi at both cells lies in the band; returns (that
        cell, reflected direction) or None."""
        axes = [k for k in range(3) if CV[i, k] != 0]
        if len(axes) != 2:
            return None
        pos = (x, y, z)
        n = (self.nx, self.ny, self.nz)

        def step(k):
            q = list(pos)
            q[k] = (q[k] + CV[i, k]) % n[k]
            return q[2], q[1], q[0]

        sa, sb = (bool(self.solid3[step(k)]) for k in axes)
        if sa == sb:
            return None
        wall, tang = (axes[0], axes[1]) if sa else (axes[1], axes[0])
        yt = step(tang)
        lo, hi = self.kw["band_lo"], self.kw["band_hi"]
        if not (lo <= f <= hi and lo <= self.phi_at(*yt) <= hi):
            return None
        cr = CV[i].copy()
        cr[wall] = -cr[wall]
        return yt, int(np.nonzero((CV == cr).all(axis=1))[0][0])

    def put_g(self, t, r, v, out):
        """Write g population r arriving at cell t, here or in a face message."""
        if self.owns(t[0]):
            self.g2[self.idx(*t), r] = v
        elif t[0] == (self.z0 - 1) % self.nz:
            assert np.isnan(out["lo_g"][DOWN.index(r), t[1], t[2]])
            out["lo_g"][DOWN.index(r), t[1], t[2]] = v
            self.reflected_across += 1
        else:
            assert np.isnan(out["hi_g"][UP.index(r), t[1], t[2]])
            out["hi_g"][UP.index(r), t[1], t[2]] = v
            self.reflected_across += 1

    def receive(self, from_below, from_above):
        """Populations streamed in by the slab below (its upward ones, into
        this slab's first plane) and the slab above (its downward ones, into
        the last plane)."""
        for (hh, gg), z, dirs in ((from_below, self.z0, UP), (from_above, self.z1 - 1, DOWN)):
            for j, i in enumerate(dirs):
                for y in range(self.ny):
                    for x in range(self.nx):
                        if not np.isnan(hh[j, y, x]):
                            self.h2[self.idx(z, y, x), i] = hh[j, y, x]
                        if not np.isnan(gg[j, y, x]):
                            self.g2[self.idx(z, y, x), i] = gg[j, y, x]

    def swap(self):
        self.h, self.g = self.h2, self.g2


def split(nz, parts):
    """Contiguous z ranges of nearly equal height."""
    edges = [round(k * nz / parts) for k in range(parts + 1)]
    return [(edges[k], edges[k + 1]) for k in range(parts)]


def run(dims, solid3, normals, theta, kw, h, g, ghost, bounds, steps, xbc=None):
    """Advance the slabs of ``bounds`` together for ``steps`` steps in one
    process; returns the reassembled h, g, ghosts and the values each slab
    sent per step."""
    slabs = [Slab(dims, z0, z1, solid3, normals, theta, kw, h, g, ghost, xbc)
             for z0, z1 in bounds]
    n = len(slabs)
    for _ in range(steps):
        for s in slabs:
            s.compute_phi()
            s.boundary_states()
        faces = [s.face_planes() for s in slabs]
        for k, s in enumerate(slabs):
            s.halo_lo = faces[(k - 1) % n][1]
            s.halo_hi = faces[(k + 1) % n][0]
        for s in slabs:
            s.update_ghosts()
        outs = [s.collide_and_stream() for s in slabs]
        for k, s in enumerate(slabs):
            below, above = outs[(k - 1) % n], outs[(k + 1) % n]
            s.receive((below["hi_h"], below["hi_g"]), (above["lo_h"], above["lo_g"]))
            s.swap()
    cat = lambda a: np.concatenate([getattr(s, a) for s in slabs])
    run.reflected_across = sum(s.reflected_across for s in slabs)
    return cat("h"), cat("g"), cat("ghost"), [s.values_sent / steps for s in slabs]


# ------------------------------------------------------------ a test case
DIMS = (10, 8, 9)
KW = dict(sigma=0.01, W=4.0, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=0.1, nu_L=0.05,
          theta_deg=60.0, blend=0.95, F_mode=1, mobility_corr=1, free_slip=1,
          band_lo=0.5, band_hi=0.95, Fex=(1e-6, 0.0, -2e-6))


def case():
    """Plates at y = 0 and y = 7 and a box obstacle that crosses slab faces;
    a drop off every mirror plane.  Returns the oracle lattice after its
    initialisation and (solid3, normals, angles, h, g, ghosts) of that
    state."""
    nx, ny, nz = DIMS
    solid3 = np.zeros((nz, ny, nx), np.uint8)
    solid3[:, 0, :] = solid3[:, -1, :] = 1
    solid3[2:7, 1:4, 6:9] = 1
    L = O.OracleLattice(nx, ny, nz, solid=solid3.reshape(-1), nthreads=1, **KW)
    phi0 = O.tanh_phi(0, DIMS, (3.3, 4.2, 4.4), 3.1, KW["W"]) * (1 - solid3.reshape(-1))
    L.init_phi(phi0)
    h, g = L.populations()
    theta = np.full(nx * ny * nz, KW["theta_deg"])
    return L, (solid3, L.normals(), theta, h, g, L.ghosts())


# ------------------------------------------------- the same over gloo ranks
def rank_main(rank, world, port, steps, out_path):
    """One slab per process; the phi planes and the face populations go
    between neighbouring ranks with point-to-point gloo messages (tags keep
    the directions apart, so two ranks that are each other's upper and
    lower neighbour still match); rank 0 writes the reassembled state."""
    import os
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, (solid3, nrm, theta, h, g, ghost) = case()
        z0, z1 = split(DIMS[2], world)[rank]
        s = Slab(DIMS, z0, z1, solid3, nrm, theta, KW, h, g, ghost)
        up, down = (rank + 1) % world, (rank - 1) % world

        def swap_msgs(to_up, to_down, tag):
            """Send arrays up and down; return (from below, from above)."""
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
            reqs, got_lo, got_hi = [], [], []
            for k, (a, b) in enumerate(zip(to_up, to_down)):
                lo, hi = torch.empty(a.shape, dtype=torch.float64), torch.empty(
                    b.shape, dtype=torch.float64)
                reqs += [dist.isend(t(a), up, tag=tag + 2 * k),
                         dist.isend(t(b), down, tag=tag + 2 * k + 1),
                         dist.irecv(lo, down, tag=tag + 2 * k),
                         dist.irecv(hi, up, tag=tag + 2 * k + 1)]
                got_lo.append(lo)
                got_hi.append(hi)
            for r in reqs:
                r.wait()
            return [x.numpy() for x in got_lo], [x.numpy() for x in got_hi]

        for _ in range(steps):
            s.compute_phi()
            s.boundary_states()
            first, last = s.face_planes()
            (s.halo_lo,), (s.halo_hi,) = swap_msgs([last], [first], 10)
            s.update_ghosts()
            out = s.collide_and_stream()
            below, above = swap_msgs([out["hi_h"], out["hi_g"]], [out["lo_h"], out["lo_g"]], 20)
            s.receive(tuple(below), tuple(above))
            s.swap()
        parts = [None] * world
        dist.all_gather_object(parts, (s.h, s.g, s.ghost, s.values_sent / steps))
        if rank == 0:
            np.savez(out_path, h=np.concatenate([p[0] for p in parts]),
                     g=np.concatenate([p[1] for p in parts]),
                     ghost=np.concatenate([p[2] for p in parts]),
                     sent=np.array([p[3] for p in parts]))
    finally:
        dist.destroy_process_group()
