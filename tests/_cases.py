"""Shared set-up of parity cases: the same geometry, parameters and initial
state given to the CUDA library (through the C ABI binding) and to the FP64
oracle.  Inputs come from ``synth``; neither side's output feeds the other."""
from __future__ import annotations

import os

import numpy as np

import synth

NTHREADS = os.cpu_count() or 1

ORACLE_KEYS = ("sigma", "W", "M", "rho_H", "rho_L", "nu_H", "nu_L", "theta_deg", "Fex", "gamma",
               "phi_M", "phi_m", "D", "eps", "blend", "band_lo", "band_hi", "F_tilde",
               "F_width", "F_mode", "mobility_corr", "free_slip")


def make_pair(geom: synth.Geometry, params: dict, init: dict, storage="fp64", kernel=0,
              tile=None, use_normals=True, use_theta=True, P0=0.0):
    """Return (gpu_lattice, oracle_lattice) initialised identically."""
    import oracle as O
    from paper_2512_01032_gb300 import pflb

    nrm = geom.normals() if use_normals else None
    th = geom.theta() if use_theta else None
    fr = geom.solid_frac()
    gp = dict(params)
    G = pflb.Lattice(geom.nx, geom.ny, geom.nz, solid=geom.solid, wall_normal=nrm,
                     theta_cells=th, storage=storage, solid_frac=fr, **gp)
    if tile is not None:
        G.set_kernel(kernel, *tile)
    else:
        G.set_kernel(kernel)
    op = {k: v for k, v in gp.items() if k in ORACLE_KEYS}
    Orc = O.OracleLattice(geom.nx, geom.ny, geom.nz, solid=geom.solid, wall_normal=nrm,
                          theta_cells=th, nthreads=NTHREADS, solid_frac=fr, **op)
    shape = init.get("shape", 0)
    G.init_tanh(shape, init["center"], init.get("R", 0.0), init.get("normal"), P0)
    phi0 = O.tanh_phi(shape, (geom.nx, geom.ny, geom.nz), init["center"], init.get("R", 0.0),
                      params.get("W", 4.0), normal=init.get("normal", (1.0, 0.0, 0.0)))
    phi0 = phi0 * (1 - geom.solid)
    Orc.init_phi(phi0, P0)
    return G, Orc


def rel_errors(gpu: dict, ref: dict, p_scale: float):
    """Relative infinity-norm errors of phi and P (P normalised by
    max(|P_ref|_inf, p_scale)) and the absolute infinity-norm error of u."""
    e = {}
    e["phi"] = np.max(np.abs(gpu["phi"] - ref["phi"])) / max(np.max(np.abs(ref["phi"])), 1e-300)
    e["P"] = np.max(np.abs(gpu["P"] - ref["P"])) / max(np.max(np.abs(ref["P"])), p_scale)
    e["u_abs"] = max(np.max(np.abs(gpu[k] - ref[k])) for k in ("ux", "uy", "uz"))
    return e


def gpu_fields(G):
    return {k: G.read(k) for k in ("phi", "P", "ux", "uy", "uz")}


def droplet_case(n=32, R=8.0):
    g, p, init = synth.static_droplet(n, R)
    return g, p, init


def sessile_case(n=32, theta=60.0):
    g, p, init = synth.sessile_sphere(n, theta)
    return g, p, init


def slit_case(nx=96, ny=16, nz=4, reservoir=24, force=(1e-8, 0.0, 0.0)):
    g, p, init = synth.slit(nx, ny, nz, reservoir)
    p = dict(p)
    p["Fex"] = force
    return g, p, init


def channel_case(nx=40, ny=14, nz=12, theta=120.0):
    g = synth.square_channel(nx, ny, nz, theta)
    p = synth.sessile_sphere_params(theta)
    p = dict(p, Fex=(2e-8, 0.0, 0.0), nu_L=0.2, nu_H=0.05)
    init = dict(shape=0, center=(nx / 4.0, ny / 2.0 - 0.5, nz / 2.0 - 0.5), R=0.35 * ny)
    return g, p, init
