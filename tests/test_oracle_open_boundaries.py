"""Open x boundaries of the oracle (reading R22: Dirichlet pressure with
Neumann velocity and phi, and velocity inlets, Sec. IV A) pinned to
closed forms of steady channel flow: plane Poiseuille flow under an imposed
pressure difference, and flux conservation from a velocity inlet to a
pressure outlet."""
import os

import numpy as np
import pytest

import oracle as O

NX, NY = 40, 18                        # plates: solid rows y = 0 and y = 17
H = NY - 2                             # gap between the halfway walls
MU = 1.0 / 6.0                         # rho_H nu_H with the liquid filling the channel


def _channel(lo, hi, steps):
    solid = np.zeros((1, NY, NX), np.uint8)
    solid[:, 0, :] = 1
    solid[:, -1, :] = 1
    L = O.OracleLattice(NX, NY, 1, solid=solid.reshape(-1), nthreads=os.cpu_count() or 1,
                        sigma=0.01, W=4.0, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=MU, nu_L=0.1)
    L.init_phi((1 - solid).reshape(-1).astype(float))
    L.set_x_boundaries(lo, hi)
    L.step(steps)
    m = L.macros()
    return {k: v.reshape(NY, NX) for k, v in m.items()}


def test_pressure_driven_poiseuille():
    """P = dP at x = 0 and 0 at x = nx-1: the interior pressure falls
    linearly with the imposed gradient dP / (nx - 1) (within 3 %), and the
    velocity profile is the parabola u = G (y - 1/2)(H + 1/2 - y) / (2 mu)
    of that gradient (within 2 % of its maximum)."""
    dP = 2e-3
    m = _channel(dict(type="pressure", P=dP), dict(type="pressure", P=0.0), 8000)
    P = m["P"][1:-1, :].mean(axis=0)
    xs = np.arange(5, NX - 5)
    G = -np.polyfit(xs, P[xs], 1)[0]
    assert G == pytest.approx(dP / (NX - 1), rel=0.03)
    y = np.arange(1, NY - 1)
    want = G * (y - 0.5) * (H + 0.5 - y) / (2 * MU)
    got = m["ux"][1:-1, NX // 2]
    assert np.max(np.abs(got - want)) < 0.02 * want.max(), (got, want)
    # no transverse flow, and the same flux through every interior section
    assert np.max(np.abs(m["uy"][1:-1, 2:-2])) < 1e-3 * want.max()
    flux = m["ux"][1:-1, 2:-2].sum(axis=0)
    assert np.ptp(flux) < 1e-3 * flux.mean()


def test_velocity_inlet_to_pressure_outlet():
    """A uniform inlet velocity U at x = 0 (phi = 1) and P = 0 at x = nx-1:
    every interior cross-section carries the same flux (steady mass
    conservation, to 1e-3), which is the inlet flux U H within 5 % (the
    equilibrium inlet is first-order: the adjacent node's non-equilibrium
    part is not reconstructed, and at H = 16 the inflow falls 3.6 % short),
    the profile develops towards the parabola of that flux, and the pressure
    falls towards the outlet."""
    U = 5e-3
    m = _channel(dict(type="velocity", u=(U, 0.0, 0.0), phi=1.0),
                 dict(type="pressure", P=0.0), 8000)
    flux = m["ux"][1:-1, 2:-2].sum(axis=0)
    assert np.ptp(flux) < 1e-3 * flux.mean()
    assert flux.mean() == pytest.approx(U * H, rel=0.05)
    U = flux.mean() / H
    y = np.arange(1, NY - 1)
    parab = 1.5 * U * (y - 0.5) * (H + 0.5 - y) / (H * H / 4.0)
    got = m["ux"][1:-1, NX - 6]
    assert np.max(np.abs(got - parab)) < 0.1 * parab.max()
    P = m["P"][1:-1, :].mean(axis=0)
    assert P[3] > P[NX // 2] > P[NX - 4] > -1e-9


def test_boundary_requests_are_checked():
    L = O.OracleLattice(8, 6, 1, sigma=0.01, W=4.0, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=0.1,
                        nu_L=0.1)
    with pytest.raises(ValueError):
        L.set_x_boundaries(dict(type="pressure", P=0.0), None)  # one side only
    L.set_x_boundaries(None, None)  # periodic again


def test_boundary_ramp_is_linear_in_steps():
    """ramp_steps: the boundary pressure goes linearly from the rest state
    (boundaries off before) to its value over the ramp, read back at the
    boundary cells; a new value mid-ramp starts from the value in effect."""
    solid = np.zeros((1, NY, NX), np.uint8)
    solid[:, 0, :] = 1
    solid[:, -1, :] = 1
    L = O.OracleLattice(NX, NY, 1, solid=solid.reshape(-1), nthreads=2, sigma=0.01, W=4.0,
                        M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=MU, nu_L=0.1)
    L.init_phi((1 - solid).reshape(-1).astype(float))
    P1 = 1e-3
    L.set_x_boundaries(dict(type="pressure", P=P1), dict(type="pressure", P=0.0), ramp_steps=40)

    def p_in():
        return L.macros()["P"].reshape(NY, NX)[NY // 2, 0]

    assert p_in() == 0.0
    L.step(10)
    assert p_in() == pytest.approx(0.25 * P1, rel=1e-12)
    L.step(30)
    assert p_in() == pytest.approx(P1, rel=1e-12)
    L.step(5)
    assert p_in() == pytest.approx(P1, rel=1e-12)
    L.set_x_boundaries(dict(type="pressure", P=0.0), dict(type="pressure", P=0.0), ramp_steps=10)
    L.step(5)
    assert p_in() == pytest.approx(0.5 * P1, rel=1e-12)


def test_boundary_cells_emit_the_equilibria_of_their_boundary_state():
    """Per cell, one whole step (reading R22): undoing push streaming (and
    halfway bounce-back at the plates) recovers what each boundary cell
    emitted, which is the equilibrium h_i = phi_b Gamma_i(u_b),
    g_i = w_i P_b / T + rho_b (Gamma_i(u_b) - w_i) of its boundary state.
    Velocity inlet (x = 0): u_b and phi_b as given, P_b = T sum g of the
    adjacent cell x = 1.  Pressure outlet (x = nx-1): P_b as given, phi_b =
    sum h and u_b = (sum c g + F/2) / rho(phi_b) of the adjacent cell
    x = nx-2 (bulk form).  All from the pre-step populations, to rounding."""
    nx, ny, nz = 24, 10, 2
    solid = np.zeros((nz, ny, nx), bool)
    solid[:, 0, :] = solid[:, -1, :] = True
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi0 = 0.5 + 0.3 * np.sin(2 * np.pi * X / nx + 0.4) * np.cos(np.pi * Y / ny)
    F = np.array([2e-6, -1e-6, 0.0])
    L = O.OracleLattice(nx, ny, nz, solid=solid.astype(np.uint8).reshape(-1), nthreads=2,
                        sigma=0.01, W=4.0, M=0.02, rho_H=1.0, rho_L=1e-3, nu_H=MU, nu_L=0.1,
                        Fex=tuple(F))
    L.init_phi((phi0 * ~solid).reshape(-1))
    u_in, phi_in, P_out = np.array([3e-3, 1e-3, 0.0]), 0.7, 1e-3
    L.set_x_boundaries(dict(type="velocity", u=tuple(u_in), phi=phi_in),
                       dict(type="pressure", P=P_out))
    L.step(5)
    h, g = L.populations()
    L.step(1)
    h1, g1 = L.populations()
    c, w, opp = O.lattice_tables()
    T = 1.0 / 3.0
    flat = solid.reshape(-1)
    worst, count = 0.0, 0
    for z in range(nz):
        for y in range(1, ny - 1):
            for x, adj in ((0, 1), (nx - 1, nx - 2)):
                cell = (z * ny + y) * nx + x
                a = (z * ny + y) * nx + adj
                if x == 0:
                    phi_b, u_b, P_b = phi_in, u_in, T * g[a].sum()
                else:
                    phi_b = h[a].sum()
                    rho_a = 1e-3 + phi_b * (1.0 - 1e-3)
                    u_b, P_b = (c.T @ g[a] + 0.5 * F) / rho_a, P_out
                rho_b = 1e-3 + phi_b * (1.0 - 1e-3)
                G = O.gamma_vec(u_b)
                want_h = phi_b * G
                want_g = w * P_b / T + rho_b * (G - w)
                for i in range(19):
                    to = (((z + c[i, 2]) % nz) * ny + (y + c[i, 1]) % ny) * nx + (x + c[i, 0]) % nx
                    got_h, got_g = (h1[cell, opp[i]], g1[cell, opp[i]]) if flat[to] else \
                        (h1[to, i], g1[to, i])
                    worst = max(worst, abs(got_h - want_h[i]), abs(got_g - want_g[i]))
                count += 1
    assert count == 2 * nz * (ny - 2)
    assert worst < 1e-15  # rounding (measured 0: the same operations)
