"""Reduced-precision population storage (FP16 weight-scaled, BF16 as is,
FP32 arithmetic) against the FP64 oracle.

Pointwise bound after n steps, derived from the formats: h_i / w_i lies in
about [0, 1], where FP16 spacing is at most 2^-11, and BF16's relative
spacing is 2^-8 at any magnitude, so each stored moving h_i is off by at
most w_i 2^-12 (FP16) or w_i 2^-9 (BF16); a cell's phi collects those of its 18 incoming populations and the
compensation of its own outgoing ones (rest population), at most
2 (1 - w_0) 2^-12 = 3.3e-4 (FP16) or 2.6e-3 (BF16) per step; the test allows
n times that.  Total phi is conserved (mass-conserving rounding of h).

Error table: the Laplace pressure jump of the static droplet, the contact
angle of a drop on a flat wall and the mass drift, for each storage format
against the FP64 oracle (target for the reduced-precision form: Laplace
pressure and contact angle within 1 % of the oracle)."""
import numpy as np
import pytest

from tests import _cases as CS

pytestmark = pytest.mark.gpu

PER_STEP = {"fp16": 2 * (2.0 / 3.0) * 2.0 ** -12, "bf16": 2 * (2.0 / 3.0) * 2.0 ** -9}


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("kernel", [0, 1])
def test_reduced_storage_pointwise_bound(storage, kernel):
    g, p, init = CS.droplet_case()
    G, Orc = CS.make_pair(g, p, init, storage=storage, kernel=kernel)
    t = 0
    for s in (1, 4, 10):
        G.step(s - t)
        Orc.step(s - t)
        t = s
        e = CS.rel_errors(CS.gpu_fields(G), Orc.macros(), 2 * p["sigma"] / init["R"])
        assert e["phi"] <= max(s, 1) * PER_STEP[storage] * 1.0001, (storage, s, e)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("nx", [36, 40])
def test_pipelined_reduced_storage_pointwise_bound(storage, nx):
    """The pipelined kernel at 16-bit storage on a walled channel with a drop
    and a body force: rows staged in 8-byte chunks (nx = 36, not a multiple
    of 8) or 16-byte chunks (nx = 40), wall nodes updated after each
    block's march; the same pointwise bound against the oracle."""
    g, p, init = CS.channel_case(nx, 14, 12)
    G, Orc = CS.make_pair(g, p, init, storage=storage, kernel=3)
    assert G.get_kernel()["kind"] == 3
    t = 0
    for s in (1, 4, 10):
        G.step(s - t)
        Orc.step(s - t)
        t = s
        e = CS.rel_errors(CS.gpu_fields(G), Orc.macros(), 2 * p["sigma"] / init["R"])
        assert e["phi"] <= max(s, 1) * PER_STEP[storage] * 1.0001, (storage, nx, s, e)


def _drop_on_flat_wall(theta):
    """Quasi 2-D drop on a flat floor (72 x 1 x 30, walls z = 0 and 29, the
    lid at 90 deg), started as a half disc of radius 14: geometry, params
    and initial phi, as in the oracle's contact-angle pin."""
    nx, ny, nz, R, W = 72, 1, 30, 14.0, 4.0
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    nw = np.zeros((nz, ny, nx, 3))
    nw[1, :, :, 2] = 1
    nw[-2, :, :, 2] = -1
    th = np.full((nz, ny, nx), theta)
    th[-2] = 90.0
    p = dict(sigma=0.01, W=W, M=0.05, rho_H=1.0, rho_L=1e-3, nu_H=0.1, nu_L=0.1, blend=0.0)
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((X - 36.0) ** 2 + (Z - 0.5) ** 2)
    phi0 = (0.5 * (1 + np.tanh(2 * (R - r) / W)) * (1 - solid)).reshape(-1)
    return (nx, ny, nz), solid.reshape(-1), nw.reshape(-1), th.reshape(-1), p, phi0


def _wall_angle(phi, dims):
    """Contact angle (deg) from a circle fitted to the phi = 0.5 contour above
    the wall's diffuse layer (Sec. IV A), wall plane at z = 0.5."""
    import math
    import synth
    nx, ny, nz = dims
    phi = phi.reshape(nz, ny, nx)[:, 0, :]
    pts = synth.contour_points(phi[1:-1], 0.5)
    pts[:, 1] += 1.0
    pts = pts[pts[:, 1] > 0.5 + 2.0]
    cx, cz, rr = synth.fit_circle(pts)
    return math.degrees(math.acos(max(-1.0, min(1.0, (0.5 - cz) / rr))))


# Error table of the reduced-precision form against the FP64 oracle (the
# acceptance bar for 16-bit storage: Laplace pressure and contact angle each
# within 1 % of the oracle; FP32 is held to the parity scale).
BAR_DP = {"fp32": 1e-5, "fp16": 1e-2, "bf16": 1e-2}
BAR_ANGLE = {"fp32": 1e-5, "fp16": 1e-2, "bf16": 1e-2}
BAR_DRIFT = {"fp32": 5e-6, "fp16": 1e-4, "bf16": 1e-4}


def test_precision_error_table():
    """Laplace pressure jump of the static droplet (32^3, R = 8, 2000 steps),
    contact angle of a drop on a flat wall (60 and 120 deg, 3000 steps) and
    relative mass drift, for FP32, FP16 and BF16 storage (FP32 arithmetic),
    each against the FP64 oracle run of the same case; the table is printed
    and every entry held to its bar."""
    import os
    import oracle as O
    from paper_2512_01032_gb300 import pflb
    rows = {st: {} for st in ("fp32", "fp16", "bf16")}
    # Laplace jump
    g, p, init = CS.droplet_case()
    op = {k: v for k, v in p.items() if k in CS.ORACLE_KEYS}
    Orc = O.OracleLattice(g.nx, g.ny, g.nz, nthreads=os.cpu_count() or 1, **op)
    phi0 = O.tanh_phi(0, (g.nx, g.ny, g.nz), init["center"], init["R"], p["W"])
    Orc.init_phi(phi0)
    Orc.step(2000)
    m = Orc.macros()
    ref_dp = m["P"][m["phi"] > 0.95].mean() - m["P"][m["phi"] < 0.05].mean()
    for st in rows:
        L = pflb.Lattice(g.nx, g.ny, g.nz, storage=st, **p)
        L.init_tanh(0, init["center"], init["R"])
        d0 = L.diag()
        L.step(2000)
        d = L.diag()
        rows[st]["dp"] = (d["dp"] - ref_dp) / ref_dp
        rows[st]["drift_drop"] = (d["mass"] - d0["mass"]) / d0["mass"]
        L.close()
    # contact angle on a flat wall
    for theta in (60.0, 120.0):
        dims, solid, nw, th, pw, phi0 = _drop_on_flat_wall(theta)
        Orc = O.OracleLattice(*dims, solid=solid, wall_normal=nw, theta_cells=th,
                              nthreads=os.cpu_count() or 1, **pw)
        Orc.init_phi(phi0)
        Orc.step(3000)
        ref = _wall_angle(Orc.macros()["phi"], dims)
        for st in rows:
            L = pflb.Lattice(*dims, solid=solid, wall_normal=nw, theta_cells=th, storage=st, **pw)
            L.init_phi(phi0)
            d0 = L.diag()
            L.step(3000)
            d = L.diag()
            rows[st][f"angle{theta:.0f}"] = (_wall_angle(L.read("phi"), dims) - ref) / ref
            rows[st][f"drift_wall{theta:.0f}"] = (d["mass"] - d0["mass"]) / d0["mass"]
            L.close()
    print("relative errors against the FP64 oracle (reference dp %.6e):" % ref_dp)
    for st, r in rows.items():
        print(" ", st, {k: "%+.2e" % v for k, v in r.items()})
    for st, r in rows.items():
        assert abs(r["dp"]) <= BAR_DP[st], (st, r)
        assert abs(r["angle60"]) <= BAR_ANGLE[st] and abs(r["angle120"]) <= BAR_ANGLE[st], (st, r)
        for k in ("drift_drop", "drift_wall60", "drift_wall120"):
            assert abs(r[k]) <= BAR_DRIFT[st], (st, k, r)


@pytest.mark.slow
def test_config3_slit_filling_precision():
    """The capillary-filling slit as configured for the precision study:
    1024 x 64 x 4, walls y = 0 and 63 over 128 <= x < 896 (theta = 45),
    liquid filling the left reservoir, density ratio 1000, viscosity ratio
    50 (nu_H = 1/60), sigma = 0.01, W = 4, 100 000 steps.  The penetration
    length l(t) (the device front probe, phi = 0.5 crossing along x in the
    channel's centre rows) every 5000 steps at each storage against FP64
    storage on the GPU, which stands in for the oracle here (parity with it
    per step is 1e-11, 1e-10 in wall cases; the oracle itself would need
    about 45 minutes on 16 host cores for this run).  The slit fills until
    the reservoir's 128 cells of liquid are used up (l ~ 190 after 35 000
    steps) and then rests.
    Measured: l(t) within 2.5e-4 (FP32), 2.2e-3 (FP16) and 2.6e-2 (BF16) of
    FP64; relative mass drift 5.8e-5 (FP32, no compensation), -4.2e-4 (FP16:
    the gas phase's populations sit below FP16's normal range and the
    rounding compensation cannot hold them), 1.4e-7 (BF16).  BF16 misses
    the 1 % target on this case: it lags during the fast filling (107.8
    against 110.6 at 15 000 steps) and rests 1.5 % further in with spurious
    currents four times FP64's.  The bars below hold FP32 and FP16 to their
    formats and record BF16's shortfall without calling it a pass of the
    1 % target."""
    import synth
    from paper_2512_01032_gb300 import pflb
    g, p, init = synth.slit(1024, 64, 4, 128)
    runs = {}
    for st in ("fp64", "fp32", "fp16", "bf16"):
        L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                         theta_cells=g.theta(), storage=st, **p)
        L.init_tanh(init["shape"], init["center"], init["R"], init["normal"])
        L.set_region((128, 896, 31, 33, 0, g.nz))
        m0 = L.diag()["mass"]
        ls = []
        for _ in range(20):
            L.step(5000)
            d = L.diag()
            ls.append(d["front_x"] - 127.0)
        runs[st] = (np.array(ls), (d["mass"] - m0) / m0)
        L.close()
    ref, drift64 = runs["fp64"]
    assert abs(drift64) < 1e-12
    assert ref[0] > 5 and 150 < ref[-1] < 230
    err = {st: np.max(np.abs(runs[st][0] - ref) / ref) for st in ("fp32", "fp16", "bf16")}
    drift = {st: abs(runs[st][1]) for st in ("fp32", "fp16", "bf16")}
    assert err["fp32"] < 1e-3 and drift["fp32"] < 2e-4, (err, drift)
    assert err["fp16"] < 1e-2 and drift["fp16"] < 1e-3, (err, drift)
    assert err["bf16"] < 5e-2 and drift["bf16"] < 1e-6, (err, drift)
