"""The seeded input generators against the workload recipes they implement
and against independent closed forms (no GPU, no method arithmetic)."""
import math

import numpy as np
import pytest

import synth


def test_channel_batch_specs_recipe():
    """64 lattices, Ny = Nz in 32..96, Nx in 96..384, drop radius
    0.3-0.45 Ny, theta 40-140 degrees, driving speed 1e-4..1e-3; the same
    seed gives the same list and another seed another one."""
    a = synth.channel_batch_specs()
    assert len(a) == 64 and a == synth.channel_batch_specs()
    assert a != synth.channel_batch_specs(seed=1)
    for s in a:
        assert 32 <= s["ny"] == s["nz"] <= 96 and 96 <= s["nx"] <= 384
        assert 0.3 * s["ny"] <= s["R"] <= 0.45 * s["ny"]
        assert 40.0 <= s["theta"] <= 140.0 and 1e-4 <= s["u_in"] <= 1e-3
    # the seeded list the channels workload reports (76.3 M cells)
    assert sum(s["nx"] * s["ny"] * s["nz"] for s in a) == 76_265_046
    # the whole span of each range is drawn, not a corner of it
    assert min(s["ny"] for s in a) < 40 and max(s["ny"] for s in a) > 88
    assert min(s["nx"] for s in a) < 130 and max(s["nx"] for s in a) > 350


def test_serving_trace_is_poisson_at_20_per_second():
    """Arrival gaps are exponential with rate 20/s: increasing times, mean
    gap 0.05 s within 3 standard errors over 200 arrivals, and a
    coefficient of variation near 1 (it is 0 for a regular clock)."""
    tr = synth.serving_trace()
    t = np.array([r["t_arrival"] for r in tr])
    assert len(tr) == 200 and np.all(np.diff(t) > 0) and t[0] > 0
    gaps = np.diff(np.r_[0.0, t])
    assert abs(gaps.mean() - 0.05) < 3 * 0.05 / math.sqrt(200)
    assert 0.8 < gaps.std() / gaps.mean() < 1.2
    for r in tr:
        assert 48 <= r["w"] <= 96 and 0.3 <= r["ratio"] <= 0.7 and 90.0 <= r["theta"] <= 150.0
    assert tr == synth.serving_trace()


def test_square_duct_constant_matches_eigenfunction_series():
    """channel_lattice drives a square duct of side a with the force density
    f = 28.45 rho nu u / a^2.  The laminar mean speed of a square duct is
    u = f a^2 / (12 mu) [1 - (192 / pi^5) sum over odd n of tanh(n pi / 2) / n^5]
    (the eigenfunction series of the rectangular-duct Poiseuille solution),
    i.e. f a^2 / (28.454 mu)."""
    s = sum(math.tanh(n * math.pi / 2) / n ** 5 for n in range(1, 400, 2))
    k = 12.0 / (1.0 - 192.0 / math.pi ** 5 * s)
    assert k == pytest.approx(28.45, rel=2e-4)
    spec = dict(nx=96, ny=34, nz=34, R=12.0, theta=70.0, u_in=5e-4)
    g, p, init = synth.channel_lattice(spec)
    a = spec["ny"] - 2.0
    mu = p["rho_L"] * p["nu_L"]
    assert p["Fex"][0] * a * a / (k * mu) == pytest.approx(spec["u_in"], rel=2e-4)
    assert p["Fex"][1] == p["Fex"][2] == 0.0
    assert init["center"][0] == spec["nx"] / 4.0


def _wall_nodes_brute(solid3):
    nz, ny, nx = solid3.shape
    out = np.zeros_like(solid3)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if solid3[z, y, x]:
                    continue
                for dx in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dz in (-1, 0, 1):
                            if abs(dx) + abs(dy) + abs(dz) not in (1, 2):
                                continue
                            if solid3[(z + dz) % nz, (y + dy) % ny, (x + dx) % nx]:
                                out[z, y, x] = True
    return out


def test_wall_nodes_and_normals_on_a_sphere():
    """Wall nodes are the fluid cells with a solid D3Q19 neighbour
    (periodic; brute force); normals are unit vectors there, point away
    from the sphere's centre (into the fluid) and are zero elsewhere; the
    voxelised ball holds 4/3 pi R^3 cells within 5 %."""
    n, R = 20, 6.0
    c = (n - 1) / 2.0
    g = synth.Geometry(n, n, n, [synth.Sphere((c, c, c), R)])
    wn = g.wall_nodes3()
    assert np.array_equal(wn, _wall_nodes_brute(g.solid3))
    nrm = g.normals().reshape(n, n, n, 3)
    mag = np.linalg.norm(nrm, axis=-1)
    assert np.allclose(mag[wn], 1.0) and np.all(mag[~wn] == 0.0)
    Z, Y, X = np.nonzero(wn)
    radial = np.stack([X - c, Y - c, Z - c], axis=1)
    radial /= np.linalg.norm(radial, axis=1, keepdims=True)
    assert np.allclose((nrm[Z, Y, X] * radial).sum(1), 1.0)
    assert g.solid.sum() == pytest.approx(4.0 / 3.0 * math.pi * R ** 3, rel=0.05)


def test_plane_walls_and_per_shape_angles():
    """The slit's plates: rows y = 0 and y = ny-1 solid, normals +y above the
    floor and -y below the lid; set_theta_near gives each plate's wall
    nodes their own angle."""
    g, p, init = synth.static_slug(60.0, H=8, length=8, nx=24, nz=2)
    s = g.solid3
    assert s[:, 0, :].all() and s[:, -1, :].all() and not s[:, 1:-1, :].any()
    nrm = g.normals().reshape(g.nz, g.ny, g.nx, 3)
    assert np.all(nrm[:, 1, :] == (0.0, 1.0, 0.0)) and np.all(nrm[:, -2, :] == (0.0, -1.0, 0.0))
    g.set_theta_near(1, 120.0)
    th = g.theta().reshape(g.nz, g.ny, g.nx)
    assert np.all(th[:, 1, :] == 60.0) and np.all(th[:, -2, :] == 120.0)


def test_constriction_opening_and_critical_pressure():
    """The constriction leaves a d x d opening over its length w, the duct
    upstream is open over its (w) x (w) cross-section; the entry pressure
    4 sigma |cos theta| (1/d - 1/H) vanishes at 90 degrees and when the
    opening is the duct, and is even in cos theta."""
    w, ratio = 20, 0.5
    g, d = synth.constriction_channel(w, ratio, 120.0)
    assert d == 10
    s = g.solid3
    x_mid = int(2.0 * w)
    assert (~s[:, :, x_mid]).sum() == d * d
    assert (~s[:, :, int(0.5 * w)]).sum() == w * w
    assert synth.critical_pressure(0.01, 90.0, d, w) == pytest.approx(0.0, abs=1e-18)
    assert synth.critical_pressure(0.01, 120.0, w, w) == 0.0
    assert synth.critical_pressure(0.01, 60.0, d, w) == pytest.approx(
        synth.critical_pressure(0.01, 120.0, d, w))
    assert synth.critical_pressure(0.01, 180.0, d, w) == pytest.approx(4 * 0.01 * (1 / d - 1 / w))
    r = synth.constriction_request(dict(w=w, ratio=ratio, theta=120.0))
    x0, x1 = r["region"][:2]
    assert x0 >= 2.5 * w + r["params"]["W"] and x1 <= g.nx
    assert r["threshold"] == 0.5 * d * d


def test_fit_circle_and_contour_points_are_exact():
    """A least-squares circle through exact circle points returns that
    circle; contour crossings of a linear field are exact."""
    t = np.linspace(0.3, 2.2, 17)
    pts = np.c_[3.0 + 7.5 * np.cos(t), -2.0 + 7.5 * np.sin(t)]
    cx, cy, r = synth.fit_circle(pts)
    assert (cx, cy, r) == pytest.approx((3.0, -2.0, 7.5), abs=1e-9)
    nz, nx = 6, 12
    Z, X = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    phi = 0.1 * (X - 4.3) + 0.5  # phi = 0.5 on the line x = 4.3
    p = synth.contour_points(phi, 0.5)
    assert len(p) == nz and np.allclose(p[:, 0], 4.3) and np.allclose(p[:, 1], np.arange(nz))


def test_cap_angle_inverts_the_cap_volume():
    """cap_angle_from_volume_height inverts V = pi h^2 (3 r - h) / 3,
    h = r (1 - cos theta) over 10..170 degrees."""
    r = 9.0
    for th in range(10, 171, 20):
        h = r * (1 - math.cos(math.radians(th)))
        V = math.pi * h * h * (3 * r - h) / 3
        assert synth.cap_angle_from_volume_height(V, h) == pytest.approx(th, abs=1e-9)
