"""Pins of the oracle's sub-voxel walls (reading R23: walls that cut fluid
cells, the volume-weighted sampling of Sec. II B and the offset walls of
Sec. IV A).

- the voxel limit: with every solid fraction 0 or 1 the oracle is the voxel
  rule of R6, bit for bit;
- the sample and the ghost links on a field linear along the wall normal:
  phi_smpl is the volume average of the parallelepiped standing on the wall,
  (1 - s) phi(x) + s phi(x + c_n), which on a linear field is phi at the
  parallelepiped's centroid; links into solid cells and links into cut cells
  that point into the wall carry ghosts (links parallel to the wall do not
  cross it), and with no tangential gradient w = -cos(theta) n_w (R8);
- a planar interface meeting an offset wall at 90 degrees: every ghost, and
  every stencil value s_y phi_{s,i} + (1 - s_y) phi(y), is the tanh profile
  of Eq. 12 continued to the neighbour, so the wall nodes see the bulk.
"""
import math

import numpy as np
import pytest

import oracle as O

W = 4.0


def _slit(nx=8, ny=10, nz=4, s=0.3):
    """Solid rows y = 0 and y = ny - 1, cut rows y = 1 and y = ny - 2 with
    solid fraction s (the walls sit s into those cells), wall normals +-y."""
    N = nx * ny * nz
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, 0, :] = solid[:, ny - 1, :] = 1
    frac = np.zeros((nz, ny, nx))
    frac[:, 1, :] = frac[:, ny - 2, :] = s
    nrm = np.zeros((nz, ny, nx, 3))
    nrm[:, : ny // 2, :, 1] = 1.0
    nrm[:, ny // 2:, :, 1] = -1.0
    return solid.reshape(-1), frac.reshape(-1), nrm.reshape(N, 3)


def _lattice(solid, frac, nrm, nx=8, ny=10, nz=4, **kw):
    p = dict(sigma=0.01, W=W, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=0.1, nu_L=0.1)
    p.update(kw)
    return O.OracleLattice(nx, ny, nz, solid=solid, wall_normal=nrm, solid_frac=frac, **p)


def test_voxel_limit_is_bitwise_the_voxel_rule():
    """Fractions of 0 on every fluid cell: 30 steps of a drop on the walls
    with blend and mobility correction equal the run without fractions."""
    nx, ny, nz = 12, 10, 6
    solid, _, nrm = _slit(nx, ny, nz)
    zero = np.zeros(nx * ny * nz)
    phi0 = O.tanh_phi(0, (nx, ny, nz), (5.5, 1.0, 2.5), 3.5, W) * (1 - solid)
    runs = []
    for fr in (None, zero):
        L = _lattice(solid, fr, nrm, nx, ny, nz, theta_deg=60.0, blend=0.95, free_slip=1,
                     F_mode=1)
        L.init_phi(phi0)
        L.step(30)
        runs.append((L.populations(), L.ghosts()))
    (h0, g0), gh0 = runs[0]
    (h1, g1), gh1 = runs[1]
    assert np.array_equal(h0, h1) and np.array_equal(g0, g1) and np.array_equal(gh0, gh1)


@pytest.mark.parametrize("s", [0.2, 0.5, 0.8])
def test_sample_and_ghost_links_on_a_linear_field(s):
    """phi = a + b y on the fluid cells, theta = 60 deg, blend 0: one ghost
    update.  At the cut cell (y = 1) phi_smpl = phi(1 + s), the average of
    the unit-thick layer [0.5 + s, 1.5 + s] standing on the wall; the links
    into the solid row (c_y = -1) get d_i = w . c_i = cos(theta); the links
    to the cut row's own cells (c_y = 0) run parallel to the wall and links
    up (c_y = +1) reach plain fluid: neither carries a ghost.  At y = 2 the
    sample is phi(2) itself and only the c_y = -1 links (into the cut row,
    towards the wall) carry ghosts.  y = 3 is no wall node."""
    nx, ny, nz = 8, 10, 4
    solid, frac, nrm = _slit(nx, ny, nz, s)
    a, b, th = 0.3, 0.05, math.radians(60.0)
    L = _lattice(solid, frac, nrm, nx, ny, nz, theta_deg=60.0, blend=0.0)
    y = np.broadcast_to(np.arange(ny)[None, :, None], (nz, ny, nx)).reshape(-1)
    phi = np.where(solid == 1, 0.0, a + b * y)
    L.init_phi(phi)
    L.set_phi_field(phi)
    marker = -7.0
    L.set_ghosts(np.full((nx * ny * nz, 19), marker))
    L.update_ghosts_only()
    gh = L.ghosts().reshape(nz, ny, nx, 19)
    c, _, _ = O.lattice_tables()

    def tanh_ghost(phi_smpl, d):  # Eqs. 14-15 at the sample and distance d
        return 0.5 * (1.0 + math.tanh(math.atanh(2 * phi_smpl - 1) + 2.0 * d / W))

    at1, at2, at3 = gh[1, 1, 3], gh[1, 2, 3], gh[1, 3, 3]
    smpl1 = a + b * (1.0 + s)
    for i in range(1, 19):
        if c[i, 1] == -1:
            assert at1[i] == pytest.approx(tanh_ghost(smpl1, math.cos(th)), abs=1e-14)
            assert at2[i] == pytest.approx(tanh_ghost(a + 2 * b, math.cos(th)), abs=1e-14)
        else:
            assert at1[i] == marker and at2[i] == marker
        assert at3[i] == marker


@pytest.mark.parametrize("s", [0.25, 0.6])
def test_planar_interface_at_90_degrees_sees_the_bulk(s):
    """A flat interface across x (tanh profile of Eq. 12) meeting the offset
    walls at 90 deg: with g = 0 the velocity mu grad(phi) / (2 rho) of every
    wall node equals that of the same column in a wall-free periodic box, so
    ghosts and the cut-cell mixing reproduce the bulk stencils exactly."""
    nx, ny, nz = 24, 10, 4
    solid, frac, nrm = _slit(nx, ny, nz, s)
    x = np.broadcast_to(np.arange(nx)[None, None, :], (nz, ny, nx)).reshape(-1)
    prof = 0.5 * (1.0 + np.tanh(2.0 * (x - 11.3) / W))
    phi = np.where(solid == 1, 0.0, prof)
    L = _lattice(solid, frac, nrm, nx, ny, nz, theta_deg=90.0, blend=0.0, mobility_corr=0)
    L.init_phi(phi)
    L.set_phi_field(phi)
    L.update_ghosts_only()
    N = nx * ny * nz
    L.set_populations(np.zeros((N, 19)), np.zeros((N, 19)))
    B = O.OracleLattice(nx, 1, 1, sigma=0.01, W=W, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=0.1,
                        nu_L=0.1, theta_deg=90.0, blend=0.0, mobility_corr=0)
    B.init_phi(prof.reshape(nz, ny, nx)[0, 0])
    B.set_populations(np.zeros((nx, 19)), np.zeros((nx, 19)))
    # h = 0 too: the macros recompute phi from h, so put phi back through h_0
    hL = np.zeros((N, 19)); hL[:, 0] = phi
    L.set_populations(hL, np.zeros((N, 19)))
    hB = np.zeros((nx, 19)); hB[:, 0] = prof.reshape(nz, ny, nx)[0, 0]
    B.set_populations(hB, np.zeros((nx, 19)))
    mL, mB = L.macros(), B.macros()
    uxL = mL["ux"].reshape(nz, ny, nx)
    # away from the periodic seam of x, where the profile jumps from 1 to 0
    xs = slice(3, nx - 3)
    assert np.abs(mB["ux"][xs]).max() > 1e-5
    for yy in (1, 2, ny - 3, ny - 2):
        assert np.allclose(uxL[:, yy, xs], mB["ux"][None, xs], rtol=1e-12, atol=1e-15), yy
        assert np.allclose(mL["uy"].reshape(nz, ny, nx)[:, yy, xs], 0.0, atol=1e-15)


def test_fraction_out_of_range_is_refused():
    solid, frac, nrm = _slit()
    bad = frac.copy()
    bad[np.flatnonzero(solid == 0)[0]] = 1.0
    with pytest.raises(ValueError):
        _lattice(solid, bad, nrm)


def _macros_at_rest(L, phi, N):
    """Velocity from mu grad(phi) / (2 rho) alone: g = 0, h_0 = phi."""
    h = np.zeros((N, 19)); h[:, 0] = phi
    L.set_populations(h, np.zeros((N, 19)))
    return L.macros()


@pytest.mark.parametrize("theta", [45.0, 120.0])
def test_cut_row_limits_are_the_voxel_walls(theta):
    """The stencil weights s_y phi_{s,i} + (1 - s_y) phi(y): at the node above
    a cut row (y = 2), grad(phi) and lap(phi) (read through the velocity
    mu grad(phi) / (2 rho) with g = 0) tend, as the row's fraction s tends to
    1, to those of the same node with row 1 solid (ghosts replace phi(1)),
    and as s tends to 0 to those of a plain fluid row 1 (swapped weights
    would exchange the two limits).  phi varies along x and y, so the
    ghosts' tangential direction is exercised too."""
    nx, ny, nz = 8, 10, 4
    N = nx * ny * nz
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = (0.35 + 0.04 * yy + 0.01 * np.cos(2 * np.pi * xx / nx)).reshape(-1)

    def run(s, row1_solid=False):
        solid, frac, nrm = _slit(nx, ny, nz, s)
        if row1_solid:
            solid = solid.reshape(nz, ny, nx).copy()
            solid[:, 1, :] = solid[:, ny - 2, :] = 1
            solid = solid.reshape(-1)
            frac = np.zeros(N)
        phi = np.where(solid == 1, 0.0, base)
        L = _lattice(solid, frac, nrm, nx, ny, nz, theta_deg=theta, blend=0.0, mobility_corr=0)
        L.init_phi(phi)
        L.set_phi_field(phi)
        L.update_ghosts_only()
        m = _macros_at_rest(L, phi, N)
        return np.stack([m[k].reshape(nz, ny, nx)[:, 2, :] for k in ("ux", "uy", "uz")])

    lo, hi = run(1e-13), run(1.0 - 1e-13)
    plain, walled = run(0.0), run(0.0, row1_solid=True)
    assert np.abs(walled - plain).max() > 1e-6  # the two limits differ
    assert np.allclose(lo, plain, rtol=0, atol=1e-15)
    assert np.allclose(hi, walled, rtol=0, atol=1e-15)
