"""Pins of the oracle's non-equilibrium-extrapolation walls (zwalls = 2; the
wall treatment of App. B): the thermal Couette flow against the paper's
analytic temperature profile (App. B, with the Prandtl and Eckert numbers of
the text), its second-order convergence, the exact linear velocity, the rest
state kept exactly, the pressure match of the boundary density, the mass
that the text's literal rho_B = rho_N lets through a wall with a temperature
step, and the compressible Poiseuille flow with cross-flow acceleration
(Sec. III.A) against an independent boundary-value solution of the
Navier-Stokes-Fourier equations."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_28679_b300 import workloads as wl
from tests.util import run_oracle

CV, RG = 2.5, 1.0
CP = CV + RG  # ideal gas


def _couette(nz, U, Pr, TC=0.33, dT=0.0, eos="ideal", wall_rho=0, **kw):
    return wl.Case(name="couette", dim=3, nx=1, ny=1, nz=nz, zwalls=2, eos=eos, R=RG, cv=CV,
                   k_over_mu=CP / Pr, tau_f=0.8, tau_g=0.8, phi_central=1, uw_hi=(U, 0.0, 0.0),
                   Tw_lo=TC, Tw_hi=TC + dT, wall_rho=wall_rho, init=dict(kind="couette", rho0=3.0), **kw)


def _analytic_T(c, xi):
    # (T - T_C)/(T_H - T_C) = xi + (Pr Ec / 2) xi (1 - xi) with Pr Ec = mu U^2 / (k (T_H - T_C)):
    # T = T_C + (T_H - T_C) xi + U^2 / (2 k/mu) xi (1 - xi)
    U = c.uw_hi[0]
    return c.Tw_lo + (c.Tw_hi - c.Tw_lo) * xi + U * U / (2.0 * c.k_over_mu) * xi * (1.0 - xi)


def _steady(c, steps):
    o = run_oracle(c, steps)
    rho, u, T = o.moments()
    return o, rho, u, T


@pytest.mark.parametrize("Pr,dT", [(0.5, 0.0), (2.0, 0.0), (1.0, 0.02)])
def test_thermal_couette_matches_analytic_profile(Pr, dT):
    # Ec = U^2 / (c_p (T_H - T_C)) = 2 for dT = 0.02 (Ec infinite for equal wall temperatures)
    c = _couette(17, 0.2, Pr, dT=dT)
    o, rho, u, T = _steady(c, 4000)
    xi = np.arange(c.nz) / (c.nz - 1)
    bump = 0.2 ** 2 / (8.0 * c.k_over_mu)
    assert np.max(np.abs(T - _analytic_T(c, xi))) <= 0.01 * bump
    # a dropped viscous-heating term or wall temperature would miss by the whole bump
    assert T[c.nz // 2] - (c.Tw_lo + 0.5 * dT) == pytest.approx(bump, rel=0.01)
    # plane Couette: u_x linear between the walls, no wall-normal flow
    assert np.max(np.abs(u[0] - 0.2 * xi)) <= 1e-12
    assert np.max(np.abs(u[2])) <= 1e-12


def test_thermal_couette_converges_at_second_order():
    errs = []
    for nz, steps in [(9, 1500), (17, 4000)]:
        c = _couette(nz, 0.2, 2.0)
        _, _, _, T = _steady(c, steps)
        xi = np.arange(nz) / (nz - 1)
        errs.append(np.max(np.abs(T - _analytic_T(c, xi))))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)


@pytest.mark.parametrize("wall_rho", [0, 1, 2])
def test_rest_state_at_wall_temperature_is_kept(wall_rho):
    # uniform rho, u = 0 and T = T_W everywhere is a steady state of the walls: nothing moves
    c = wl.Case(name="rest", dim=3, nx=3, ny=2, nz=6, zwalls=2, eos="vdw", R=1.0, cv=2.5, a=9 / 245,
                b=2 / 21, k_over_mu=3.5, Tw_lo=0.4, Tw_hi=0.4, wall_rho=wall_rho,
                init=dict(kind="uniform", rho0=1.3, T0=0.4))
    o = run_oracle(c, 50)
    rho, u, T = o.moments()
    assert np.max(np.abs(rho - 1.3)) <= 1e-13
    assert np.max(np.abs(u)) <= 1e-14
    assert np.max(np.abs(T - 0.4)) <= 1e-13


def test_boundary_density_matches_the_neighbour_pressure():
    # wall_rho = 0: P(rho_B, T_W) = P(rho_N, T_N) on both walls, here for van der Waals with
    # noisy density, a body force and different wall temperatures
    c = wl.Case(name="walls", dim=3, nx=4, ny=3, nz=8, zwalls=2, eos="vdw", R=1.0, cv=2.5, a=9 / 245,
                b=2 / 21, kappa=0.01, k_over_mu=3.5, accel=(1e-5, 0.0, -1e-5), phi_central=1,
                uw_lo=(0.0, 0.01, 0.0), uw_hi=(0.02, 0.0, 0.0), Tw_lo=0.4, Tw_hi=0.43,
                init=dict(kind="couette", rho0=1.5, amp=0.02, seed=5))
    o = run_oracle(c, 30)
    rho, u, T = o.moments()
    p = o.p
    N = c.nx * c.ny
    for zb, zn, Tw, uw in [(0, 1, 0.4, c.uw_lo), (c.nz - 1, c.nz - 2, 0.43, c.uw_hi)]:
        for k in range(N):
            kb, kn = zb * N + k, zn * N + k
            PB = orc.lib().orc_eos_P(p, rho[kb], T[kb])
            PN = orc.lib().orc_eos_P(p, rho[kn], T[kn])
            assert PB == pytest.approx(PN, rel=1e-13)
            assert T[kb] == Tw
            assert np.allclose(u.reshape(3, -1)[:, kb], uw, atol=0.0, rtol=0.0)


def test_literal_neighbour_density_leaks_mass_through_a_heated_wall():
    # wall_rho = 1 (rho_B = rho_N as the text states it): with T_W != T_N the wall link carries a
    # pressure step, so the channel keeps losing mass and a wall-normal flow remains; the pressure
    # match (wall_rho = 0) settles with no flow through the walls
    lost = {}
    for wall_rho in (0, 1):
        c = _couette(17, 0.02, 1.0, dT=0.02, wall_rho=wall_rho)
        o = run_oracle(c, 3000)
        m0 = o.moments()[0].sum()
        o.step(1000)
        rho, u, T = o.moments()
        lost[wall_rho] = (m0 - rho.sum()) / m0, np.max(np.abs(u[2]))
    assert abs(lost[0][0]) <= 1e-12 and lost[0][1] <= 1e-12
    assert lost[1][0] > 1e-5 and lost[1][1] > 1e-5


def _steady_nsf_poiseuille(L, tau, kmu, TC, TH, gx, gz, mass):
    # Steady compressible Poiseuille flow between isothermal walls at z = 0 and L (Sec. III.A, cross-flow
    # acceleration), from the Navier-Stokes-Fourier equations with mu = tau P and k = (k/mu) mu, ideal gas
    # (R = 1): (mu u')' = -rho g_x, (k T')' + mu u'^2 = 0, P' = rho g_z, u_z = 0, u = 0 and T given at the
    # walls, total mass given.  Solved as a boundary-value problem, independently of the lattice.
    from scipy.integrate import solve_bvp

    def rhs(z, y):
        u, S, T, H, P, m = y
        return np.vstack([S / (tau * P), -(P / T) * gx, H / (kmu * tau * P), -S * S / (tau * P), P * gz / T, P / T])

    def bc(ya, yb):
        return np.array([ya[0], yb[0], ya[2] - TC, yb[2] - TH, ya[5], yb[5] - mass])

    z = np.linspace(0.0, L, 200)
    P0 = mass / L * TC
    y0 = np.vstack([np.zeros_like(z), np.zeros_like(z), TC + (TH - TC) * z / L, np.zeros_like(z),
                    np.full_like(z, P0), P0 / TC * z])
    sol = solve_bvp(rhs, bc, z, y0, tol=1e-10, max_nodes=100000)
    assert sol.status == 0
    return sol.sol


@pytest.mark.parametrize("ratio", [50.0, -50.0])
def test_cross_flow_poiseuille_matches_the_steady_nsf_solution(ratio):
    # streamwise g_x with the paper's wall-normal g_z = +-50 g_x between walls at T_C and T_H: u_x, T and
    # rho against the boundary-value solution of the same equations with the simulated mass.  wall_rho = 2
    # keeps the walls tight against the hydrostatic pressure gradient (density from 1.9 to 3.1 across the
    # channel); wall_rho = 0 sets P_B = P_N against it and the channel drains
    nz, tau, kmu, TC, TH, gx = 33, 0.8, 1.75, 0.33, 0.35, 1e-4
    out = {}
    for wall_rho in (2, 0):
        c = wl.Case(name="pois", dim=3, nx=1, ny=1, nz=nz, zwalls=2, eos="ideal", R=1.0, cv=2.5, k_over_mu=kmu,
                    tau_f=tau, tau_g=tau, phi_central=1, accel=(gx, 0.0, ratio * gx), Tw_lo=TC, Tw_hi=TH,
                    wall_rho=wall_rho, init=dict(kind="couette", rho0=3.0))
        threads = orc.get_threads()
        orc.set_threads(1)
        try:
            o = run_oracle(c, 25000)
        finally:
            orc.set_threads(threads)
        rho, u, T = o.moments()
        out[wall_rho] = rho, u.reshape(3, -1), T
    rho, u, T = out[2]
    z = np.arange(nz, dtype=float)
    mass = np.trapezoid(rho, z)
    ref = _steady_nsf_poiseuille(nz - 1, tau, kmu, TC, TH, gx, ratio * gx, mass)(z)
    Umax = ref[0].max()
    assert np.max(np.abs(u[2])) <= 5e-3 * Umax
    assert np.max(np.abs(u[0] - ref[0])) <= 1e-2 * Umax
    assert np.max(np.abs(T - ref[2])) <= 4e-2 * np.ptp(ref[2])
    assert np.max(np.abs(rho - ref[4] / ref[2])) <= 3e-3 * rho.mean()
    # the cross-flow acceleration matters: without it the density profile is far off
    ref0 = _steady_nsf_poiseuille(nz - 1, tau, kmu, TC, TH, gx, 0.0, mass)(z)
    assert np.max(np.abs(rho - ref0[4] / ref0[2])) > 0.1 * rho.mean()
    # with P_B = P_N a wall-normal flow of ~10 % of U remains and mass leaves the channel
    assert np.max(np.abs(out[0][1][2])) > 5e-2 * Umax
    assert out[0][0].mean() < 0.5 * rho.mean()
