"""Physics of the CUDA path against laws the paper relies on (FP32 storage,
long runs that the oracle could not afford): the Laplace pressure jump of a
static droplet, the height of a drop resting on a solid sphere for a given
input contact angle (the paper's curved-wall wetting case, Sec. II B), and
viscous capillary filling of a slit (Lucas-Washburn, Sec. IV B)."""
import math

import numpy as np
import pytest

import synth
from tests import _physics as P

pytestmark = pytest.mark.gpu


def _lattice(g, p, storage="fp32"):
    from paper_2512_01032_gb300 import pflb
    return pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                        theta_cells=g.theta(), storage=storage, **p)


def test_laplace_pressure_jump():
    """32^3 periodic box, droplet radius 8 (W = 4, density ratio 1000,
    sigma = 0.01): after 4000 steps the pressure jump between the drop's
    centre and the far corner equals 2 sigma / R_eff within 1 %, with R_eff
    the radius of a ball of the drop's volume (sum of phi).  (Larger drops
    settle below the law with the mobility correction on, in the oracle as
    on the GPU: 2.5 % at R = 10, 5.7 % at R = 18.)"""
    n, R = 32, 8.0
    g, p, init = synth.static_droplet(n, R)
    L = _lattice(g, p)
    L.init_tanh(0, init["center"], R)
    L.step(4000)
    P_ = L.read("P").reshape(n, n, n)
    phi = L.read("phi")
    reff = (3 * phi.sum() / (4 * math.pi)) ** (1 / 3)
    c0, c1 = n // 2 - 1, n // 2  # the centre lies between sites
    dp = P_[c0:c1 + 1, c0:c1 + 1, c0:c1 + 1].mean() - P_[0, 0, 0]
    want = 2 * p["sigma"] / reff
    assert abs(dp - want) / want < 0.01, (dp, want)


def _off_axis(center, dx=1e-3):
    """The drop's centre moved 1e-3 of a spacing in x.  Started exactly on
    the box's mirror planes, the 30 deg drop at FP32 went non-finite after
    about 820 steps in one build: spreading fast over the sphere (max |u|
    1e-2) it drove phi down to -3.5e-4 next to the wall, where
    rho = rho_L + phi (rho_H - rho_L) falls to 6.5e-4 and u = j / rho
    runs away; started off the planes it has stayed finite in every run.  (The
    FP64 blow-ups at 120 and 150 deg after 2-17 k steps had another cause,
    the pole of the printed mobility-correction switch, reading R4 of
    Eq. 4.)"""
    return (center[0] + dx, center[1], center[2])


def _axis_top(phi3, c):
    """Highest z where phi on the vertical axis x = y = c is 0.5 (linear
    interpolation; the axis lies between four lattice columns)."""
    i0, i1 = int(math.floor(c)), int(math.ceil(c))
    col = 0.25 * (phi3[:, i0, i0] + phi3[:, i0, i1] + phi3[:, i1, i0] + phi3[:, i1, i1])
    k = int(np.where(col >= 0.5)[0].max())
    return k + (col[k] - 0.5) / (col[k] - col[k + 1])


@pytest.mark.parametrize("theta", [30.0, 60.0, 90.0, 120.0, 150.0])
def test_drop_height_on_sphere(theta):
    """64^3: solid sphere of radius 15 centred on the floor, drop of radius
    10 set on its top; after 15000 steps the drop's top lies where a ball of
    the drop's volume meeting the sphere at the input angle puts it, within
    one lattice spacing (the diffuse interface and the voxel wall shift it by
    0.4-0.6 spacings)."""
    n = 64
    g, p, drop = synth.sessile_sphere(n, theta)
    L = _lattice(g, p)
    L.init_tanh(0, _off_axis(drop["center"]), drop["R"])
    V = L.diag()["mass"]
    L.step(15000)
    d = L.diag()
    assert d["nonfinite"] == 0 and d["u_max"] < 1e-3
    h = _axis_top(L.read("phi").reshape(n, n, n), (n - 1) / 2.0)
    want, r, _ = P.sessile_top_on_sphere(30.0 * n / 128, theta, V)
    assert abs(h - want) < 1.0, (h, want, r)


@pytest.mark.parametrize("theta", [30.0, 60.0, 90.0, 120.0, 150.0])
def test_sessile_drop_on_sphere_128_full_run(theta):
    """The curved-wall workload at its full size: 128^3, a drop of radius 20
    on a solid sphere of radius 30, density ratio 1000, sigma 0.005, the
    optimised model with the paper's blend 0.95 and mobility correction,
    20000 steps at FP32.  Every angle stays finite and the drop's top ends
    within one lattice spacing of where a ball of the drop's volume meeting
    the sphere at the input angle puts it.  The 30 deg drop spreads slowest:
    its top is still 1.15 spacings high at 20000 steps (max |u| 3e-4), meets
    the closed form near 34000 and creeps on to -0.6 at 60000 (max |u| 8e-5,
    the steps shrinking by a quarter every 5000), so it runs 60000 steps.
    At 120 deg the contact line does not come to rest: a wall node at the
    line sits at phi ~ 0.21, the edge phi_m = 0.2 of the mobility
    correction's window (Eq. 4, switched over D = 1e-4 in phi), and with the
    ghosts lagged by the 0.95 blend the switch and the wetting condition keep
    a steady oscillation (max |u| about 6e-3, in FP64 alike); the shape
    still settles."""
    n = 128
    g, p, drop = synth.sessile_sphere(n, theta)
    L = _lattice(g, p)
    L.init_tanh(0, _off_axis(drop["center"]), drop["R"])
    V = L.diag()["mass"]
    L.step(60000 if theta == 30.0 else 20000)
    d = L.diag()
    assert d["nonfinite"] == 0
    assert d["u_max"] < (1e-2 if theta == 120.0 else 1e-3)
    h = _axis_top(L.read("phi").reshape(n, n, n), (n - 1) / 2.0)
    want, r, _ = P.sessile_top_on_sphere(30.0, theta, V)
    print("SESSILE128", theta, "top", h, "closed form", want, "u_max", d["u_max"])
    assert abs(h - want) < 1.0, (h, want, r)


def test_lucas_washburn_filling():
    """Slit of height H = 16 (walls y = 0, 17 over 128 <= x < 896, periodic
    1024 x 18 x 4 box), theta = 45, density ratio 1000, nu_H = 1/6 so that
    the viscous time H^2 / nu_H (1.5e3 steps) is short against the run:
    the front speed stays within 0.65-1.0 of the viscous balance
    [mu1 z + mu2 (L - z)] dz/dt = sigma cos(theta) H / 6 from 5e3 to 5.8e4
    steps and approaches it (the deficit is the dynamic contact angle and
    the entrance loss, which the balance leaves out)."""
    g, p, init = synth.slit(1024, 18, 4, 128)
    p = dict(p, nu_H=1.0 / 6.0)
    L = _lattice(g, p)
    L.init_tanh(init["shape"], init["center"], init["R"], init["normal"])
    mu1, mu2 = p["rho_H"] * p["nu_H"], p["rho_L"] * p["nu_L"]

    # front position from the device diagnostics (phi = 0.5 crossing along
    # +x in the two centre rows of the channel), measured from x = 127
    L.set_region((128, 896, 8, 10, 0, g.nz))

    def front():
        return L.diag()["front_x"] - 127.0

    L.step(5000)
    zs, ts = [front()], [5000]
    while ts[-1] < 58000:
        L.step(1000)
        zs.append(front())
        ts.append(L.t)
    ratios = []
    for k in range(len(zs) - 1):
        v = (zs[k + 1] - zs[k]) / (ts[k + 1] - ts[k])
        z = 0.5 * (zs[k] + zs[k + 1])
        ratios.append(v / P.washburn_speed(z, p["sigma"], p["theta_deg"], 16.0, mu1, mu2,
                                           768.0))
    assert all(0.65 < q < 1.0 for q in ratios), ratios
    assert np.mean(ratios[-10:]) > np.mean(ratios[:10])
    assert 80.0 < zs[-1] < 120.0


@pytest.mark.parametrize("theta", [20.0, 40.0, 60.0, 90.0, 120.0, 140.0, 160.0])
def test_static_slug_between_plates(theta):
    """Liquid slug at rest between flat plates 32 cells apart (192 x 34 x 4,
    periodic in x and z): after 20000 steps each meniscus is a circular arc
    meeting the plates at the input angle (circle fit to the phi = 0.5
    contour, within 2 degrees; flat at 90 degrees), the pressure jump has
    the sign and, within 10 %, the size of -2 sigma cos(theta) / H (it
    settles about 6 % below it, as the Laplace jump of large drops does),
    and the spurious currents stay below 1e-3."""
    g, p, init = synth.static_slug(theta)
    L = _lattice(g, p)
    L.init_tanh(init["shape"], init["center"], init["R"], init["normal"])
    L.step(20000)
    d = L.diag()
    assert d["nonfinite"] == 0 and d["u_max"] < 1e-3
    phi = L.read("phi").reshape(g.nz, g.ny, g.nx)[0]
    sub = phi[1:g.ny - 1, g.nx // 2:]
    pts = synth.contour_points(sub, 0.5)
    pts[:, 0] += g.nx // 2
    pts[:, 1] += 1.0
    core = pts[(pts[:, 1] > 3.5) & (pts[:, 1] < g.ny - 4.5)]  # W/2 off the plates
    H = g.ny - 2
    if theta == 90.0:
        assert np.ptp(core[:, 0]) < 0.05
        assert abs(d["dp"]) < 1e-5
        return
    cx, cy, r = synth.fit_circle(core)
    c = min(1.0, (H / 2.0) / r)
    wetting = cx > core[:, 0].mean()  # centre of curvature on the gas side
    got = math.degrees(math.acos(c)) if wetting else 180.0 - math.degrees(math.acos(c))
    assert abs(got - theta) < 2.0, got
    want = -2 * p["sigma"] * math.cos(math.radians(theta)) / H
    assert 0.9 < d["dp"] / want < 1.02, (d["dp"], want)


def _menisci(phi2, H):
    """Rear and front menisci of the slug (phi2: [y, x] at one z): for each,
    the x of the phi = 0.5 crossing on every row, a circle fit through the
    rows W/2 off the plates, and the contact angle inside the liquid."""
    ny, nx = phi2.shape
    col = phi2[1:ny - 1].mean(axis=0)
    liquid = np.where(col >= 0.5)[0]
    x_rear, x_front = liquid.min(), liquid.max()
    out = []
    for side, x0 in (("rear", x_rear), ("front", x_front)):
        lo, hi = max(0, x0 - 24), min(nx, x0 + 25)
        pts = synth.contour_points(phi2[1:ny - 1, lo:hi], 0.5)
        pts[:, 0] += lo
        pts[:, 1] += 1.0
        pts = pts[(pts[:, 1] > 3.5) & (pts[:, 1] < ny - 4.5)]
        cx, cy, r = synth.fit_circle(pts)
        xm = pts[:, 0].mean()
        c = min(1.0, (H / 2.0) / r)
        # liquid side of this meniscus: +x for the rear one, -x for the front one
        centre_in_liquid = (cx > xm) if side == "rear" else (cx < xm)
        ang = 180.0 - math.degrees(math.acos(c)) if centre_in_liquid else math.degrees(math.acos(c))
        out.append((xm, ang))
    return out


def test_dynamic_slug_in_a_slit():
    """A slug pushed along a hydrophobic slit (theta 133) by a gas velocity
    inlet against a pressure outlet (open x boundaries), with the pressure
    split of Table I measured along it: it advances, its
    front (advancing) meniscus is steeper than the static angle and its rear
    (receding) one flatter by several degrees (measured 141.8 and 124.8 at
    Ca ~ 1e-2), and the pressure falls across it.  Its speed over a
    1e4-step window (3.9e-3) is not the gas flux behind it (1.5e-3 x H): in
    the pressure-based scheme the light phase (rho = 1e-3) compresses in the
    velocity sense, div u ~ -(dP/dt) / (rho c_s^2), so the gas column acts as
    a soft spring and is not pinned here."""
    U, H = 2e-3, 32
    g, p, init, inlet, outlet = synth.dynamic_slug(U=U, H=H)
    L = _lattice(g, p)
    L.set_x_boundaries(inlet, outlet, ramp_steps=2000)
    L.init_tanh(init["shape"], init["center"], init["R"], init["normal"])
    L.step(20000)
    phi = L.read("phi").reshape(g.nz, g.ny, g.nx)[0]
    (xr0, _), (xf0, _) = _menisci(phi, H)
    L.step(10000)
    d = L.diag()
    assert d["nonfinite"] == 0
    phi = L.read("phi").reshape(g.nz, g.ny, g.nx)[0]
    (xr1, th_r), (xf1, th_a) = _menisci(phi, H)
    v = 0.5 * ((xr1 - xr0) + (xf1 - xf0)) / 10000.0
    P = L.read("P").reshape(g.nz, g.ny, g.nx)[0, g.ny // 2]
    dP = P[int(xr1) - 16] - P[int(xf1) + 16]
    ux = L.read("ux").reshape(g.nz, g.ny, g.nx)[0]
    xg = int(xr1) // 2  # gas between the inlet and the slug
    u_flux = ux[1:-1, xg].sum() / H
    print("DYNSLUG speed", v, "U", U, "delivered", u_flux, "advancing", th_a, "receding", th_r,
          "dP", dP)
    assert v > 0.5 * U
    assert th_a > 133.0 + 3.0 and th_r < 133.0 - 3.0
    assert dP > 0

    # The pressure split of Sec. III A (Table I): gas pressure ahead of the
    # front meniscus P_a, liquid behind it P_a,slug, liquid ahead of the rear
    # meniscus P_r,slug, gas behind it P_r, as cross-section means 12 cells
    # from each meniscus (phi uniform over the section there); the total
    # P_r - P_a is dP_wall + dP_a + dP_r by construction.
    Pm = L.read("P").reshape(g.nz, g.ny, g.nx)[0, 1:-1].mean(axis=0)
    xa, xb = int(xf1), int(xr1)
    Pa, Pas, Prs, Pr = Pm[xa + 12], Pm[xa - 12], Pm[xb + 12], Pm[xb - 12]
    dP_a, dP_r, dP_wall = Pas - Pa, Pr - Prs, Prs - Pas
    sigma = p["sigma"]
    lap_a = -2.0 * sigma * math.cos(math.radians(th_a)) / H  # liquid minus gas pressure
    lap_r = 2.0 * sigma * math.cos(math.radians(th_r)) / H   # gas minus liquid pressure
    xs = np.arange(xb + 12, xa - 12)
    slope = np.polyfit(xs, Pm[xs], 1)[0]
    pois = 12.0 * p["rho_H"] * p["nu_H"] * v / H ** 2  # plane Poiseuille gradient at the slug speed
    print("DYNSLUG split dP_a", dP_a, "Laplace", lap_a, "dP_r", dP_r, "Laplace", lap_r,
          "dP_wall", dP_wall, "gradient", -slope, "Poiseuille", pois)
    # each capillary jump is the Laplace pressure of its meniscus at the
    # measured dynamic angle (measured within 4.5 % and 2.5 %) ...
    assert abs(dP_a / lap_a - 1.0) < 0.10 and abs(dP_r / lap_r - 1.0) < 0.10
    # ... and the wall friction inside the slug is of the order of plane
    # Poiseuille flow at its speed, above it (1.6x measured: in a slug two
    # gaps long the flow recirculates near the menisci and dissipates more)
    assert dP_wall > 0 and 1.0 < -slope / pois < 2.5

    # Cox-Voinov (Sec. III B): theta_d^3 = theta_s^3 +- 9 Ca ln(L / l_s),
    # Ca = mu_H v / sigma.  The measured angles imply ln(L / l_s) of 45
    # (advancing) and 37 (receding); a physical slip length gives 5-15, so
    # the diffuse contact line dissipates several times more than a sharp
    # one, on both sides alike (the excess the optimised friction model of
    # Sec. III A is there to reduce).
    ca = p["rho_H"] * p["nu_H"] * v / sigma
    ts, ta, tr = (math.radians(x) for x in (133.0, th_a, th_r))
    ln_a, ln_r = (ta ** 3 - ts ** 3) / (9.0 * ca), (ts ** 3 - tr ** 3) / (9.0 * ca)
    print("DYNSLUG Cox-Voinov Ca", ca, "ln(L/l_s) advancing", ln_a, "receding", ln_r)
    assert 20.0 < ln_a < 90.0 and 20.0 < ln_r < 90.0 and 0.5 < ln_a / ln_r < 2.0


def _slug_angle(phi2, ylo, yhi, nx):
    """Contact angle of the right meniscus of a static slug between walls at
    ylo and yhi (circle fit to the phi = 0.5 contour, rows W/2 off the
    walls, inside the liquid)."""
    ny = phi2.shape[0]
    sub = phi2[1:ny - 1, nx // 2:]
    pts = synth.contour_points(sub, 0.5)
    pts[:, 0] += nx // 2
    pts[:, 1] += 1.0
    core = pts[(pts[:, 1] > ylo + 3.0) & (pts[:, 1] < yhi - 3.0)]
    cx, cy, r = synth.fit_circle(core)
    c = min(1.0, ((yhi - ylo) / 2.0) / r)
    wetting = cx > core[:, 0].mean()  # centre of curvature on the gas side
    return math.degrees(math.acos(c)) if wetting else 180.0 - math.degrees(math.acos(c))


@pytest.mark.parametrize("delta", [0.2, 0.5, 0.8])
@pytest.mark.parametrize("theta", [20.0, 60.0, 120.0, 160.0])
def test_offset_slug_angle(theta, delta):
    """The static slug between plates moved into the channel by delta (Sec.
    IV A, walls at 0.5 + delta and H + 0.5 - delta, sub-voxel reading R23),
    20000 steps at FP32: the run stays finite with bounded spurious
    currents, the meniscus keeps the wetting side of its input angle, and at
    60 and 120 deg its angle (circle fit, gap H - 2 delta) is within 8 deg
    of the input.  This light weighting does not give the paper's
    offset-independent angles (Fig. 10): measured 63.6 / 65.1 / 65.5 deg
    for 60 and 116.5 / 114.9 / 114.4 for 120 at delta 0.2 / 0.4 / 0.8, and
    32 / 37 / 41 for 20 and 149 / 143 / 141 for 160 (the cut cells evolve as
    whole fluid cells, so the wetting weakens as the wall moves into them)."""
    g, p, init = synth.offset_slug(theta, delta)
    from paper_2512_01032_gb300 import pflb
    L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                     theta_cells=g.theta(), storage="fp32", solid_frac=g.solid_frac(), **p)
    L.init_tanh(init["shape"], init["center"], init["R"], init["normal"])
    L.step(20000)
    d = L.diag()
    assert d["nonfinite"] == 0 and d["u_max"] < 5e-3
    H = g.ny - 2
    got = _slug_angle(L.read("phi").reshape(g.nz, g.ny, g.nx)[0], 0.5 + delta,
                      H + 0.5 - delta, g.nx)
    print("OFFSET", theta, delta, "angle", got, "u_max", d["u_max"])
    assert (got - 90.0) * (theta - 90.0) > 0
    if theta in (60.0, 120.0):
        assert abs(got - theta) < 8.0, got
