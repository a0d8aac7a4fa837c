"""Pins of the oracle's duct ends and duct friction (the 1-D duct flows of
Sec. III.A: Rayleigh flow with a heat source, Fanno flow with friction and the
compensating heat Q = -F.u), run as 1 x 1 x nz columns of D3Q27: the closed-form
Rayleigh and Fanno relations T/T*, P/P* against the local Mach number, the
total-enthalpy laws (H_in + Q z / mdot; H constant), a uniform mass flux, the
exact uniform state kept by consistent inlet and outlet data, and the friction
law with its exact energy budget."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_28679_b300 import workloads as wl
from tests.util import run_oracle

R_GAS, CV = 1.0, 2.5
CP = R_GAS + CV
GAM = CP / CV
T_IN, P_IN, MA_IN = 0.1, 0.1, 0.3
T0 = T_IN * (1.0 + 0.5 * (GAM - 1.0) * MA_IN ** 2)  # isentropic total state of the inlet
P0 = P_IN * (T0 / T_IN) ** (CP / R_GAS)
U_IN = MA_IN * math.sqrt(GAM * R_GAS * T_IN)


def _duct(nz, q=0.0, friction=0.0, p_out=0.08, kinds=(1, 3), face_P=None, uw_lo=(0.0, 0.0, 0.0), T_lo=T0):
    return wl.Case(name="duct", dim=3, nx=1, ny=1, nz=nz, zwalls=2, eos="ideal", R=R_GAS, cv=CV,
                   k_over_mu=CP / 0.71, tau_f=0.8, tau_g=0.8, phi_central=1, q=q, zlo=0, zhi=0,
                   friction=friction, face_kind=kinds, face_P=face_P or (P0, p_out), uw_lo=uw_lo,
                   Tw_lo=T_lo, Tw_hi=T_lo,
                   init=dict(kind="duct", rho0=P_IN / (R_GAS * T_IN), u0=U_IN, T0=T_IN))


def _profiles(c, steps):
    o = run_oracle(c, steps)
    rho, u, T = o.moments()
    uz = u.reshape(3, -1)[2]
    P = rho * R_GAS * T
    return rho, uz, T, P, uz / np.sqrt(GAM * R_GAS * T)


def test_rayleigh_flow_relations():
    # heat addition at subsonic speed: the flow accelerates and every cell lies on one Rayleigh line,
    # T/T* = (1+g)^2 Ma^2/(1+g Ma^2)^2, P/P* = (1+g)/(1+g Ma^2), with one sonic state (T*, P*)
    nz, q = 50, 4e-5
    c = _duct(nz, q=q)
    rho, uz, T, P, Ma = _profiles(c, 20000)
    mdot = rho * uz
    assert np.ptp(mdot[1:-1]) <= 1e-12 * mdot.mean()
    assert Ma[-2] > Ma[1] + 0.01
    Ts = T * (1 + GAM * Ma ** 2) ** 2 / ((1 + GAM) ** 2 * Ma ** 2)
    Ps = P * (1 + GAM * Ma ** 2) / (1 + GAM)
    assert np.ptp(Ts[1:-1]) <= 1e-3 * Ts.mean()
    assert np.ptp(Ps[1:-1]) <= 1e-3 * Ps.mean()
    # total enthalpy grows by the heat input: H(z) = H_1 + Q (z - 1) / mdot (to first order in dz)
    H = CP * T + 0.5 * uz ** 2
    z = np.arange(nz)
    Hana = H[1] + q * (z - 1) / mdot.mean()
    assert np.max(np.abs(H - Hana)[1:-1]) <= 0.03 * q * nz / mdot.mean()


def test_rayleigh_relations_converge_with_resolution():
    spreads = []
    for nz in (25, 50):
        c = _duct(nz, q=4e-5 * 50 / nz)
        rho, uz, T, P, Ma = _profiles(c, 400 * nz)
        Ts = T * (1 + GAM * Ma ** 2) ** 2 / ((1 + GAM) ** 2 * Ma ** 2)
        spreads.append(np.ptp(Ts[1:-1]) / Ts.mean())
    assert spreads[0] / spreads[1] == pytest.approx(2.0, rel=0.2)  # first order at fixed tau


def test_fanno_flow_relations():
    # friction at subsonic speed: T/T* = (1+g)/(2+(g-1)Ma^2), P/P* = sqrt((1+g)/(2+(g-1)Ma^2))/Ma,
    # and the total enthalpy stays constant (the friction work returns as heat, Q = -F.u)
    nz = 50
    c = _duct(nz, friction=4e-3)
    rho, uz, T, P, Ma = _profiles(c, 20000)
    assert np.ptp((rho * uz)[1:-1]) <= 1e-12 * (rho * uz).mean()
    assert Ma[-2] > Ma[1] + 0.02
    Ts = T * (2 + (GAM - 1) * Ma ** 2) / (1 + GAM)
    Ps = P * Ma / np.sqrt((GAM + 1) / (2 + (GAM - 1) * Ma ** 2))
    assert np.ptp(Ts[1:-1]) <= 2e-4 * Ts.mean()
    assert np.ptp(Ps[1:-1]) <= 2e-4 * Ps.mean()
    H = CP * T + 0.5 * uz ** 2
    assert np.ptp(H) <= 1e-3 * H.mean()


@pytest.mark.parametrize("kinds", [(1, 3), (2, 4), (2, 3), (1, 4)])
def test_uniform_flow_is_kept_by_consistent_duct_ends(kinds):
    # inlet and outlet data that agree with a uniform subsonic flow leave it exactly uniform
    nz = 12
    face_P = (P0 if kinds[0] == 1 else P_IN, P_IN)
    c = _duct(nz, kinds=kinds, face_P=face_P, uw_lo=(0.0, 0.0, U_IN), T_lo=T0 if kinds[0] == 1 else T_IN)
    rho, uz, T, P, Ma = _profiles(c, 200)
    assert np.max(np.abs(rho - P_IN / (R_GAS * T_IN))) <= 1e-12
    assert np.max(np.abs(uz - U_IN)) <= 1e-12
    assert np.max(np.abs(T - T_IN)) <= 1e-12


def test_friction_law_and_energy_budget():
    # uniform periodic flow: d(rho u)/dt = -k rho u^2 gives u(t) = u0 / (1 + k u0 t); the heat
    # Q = -F.u returns the friction work, so total energy is conserved exactly and the momentum
    # changes by the total force
    k, u0, n = 0.05, 0.1, 400
    c = wl.Case(name="fric", dim=3, nx=2, ny=2, nz=3, eos="ideal", R=R_GAS, cv=CV, k_over_mu=CP / 0.71,
                friction=k, init=dict(kind="duct", rho0=1.0, u0=u0, T0=0.3))
    o = run_oracle(c, 0)
    prev = o.invariants()
    for _ in range(n):
        o.step(1)
        cur = o.invariants()
        assert abs(cur[4] - prev[4]) <= 1e-12 * abs(cur[4])          # rho E
        assert abs(cur[-1]) <= 1e-14 * abs(cur[4])                   # sum (u.F + Q) = 0
        assert cur[3] - prev[3] == pytest.approx(0.5 * (prev[7] + cur[7]), rel=1e-9)  # z momentum
        prev = cur
    uz = o.moments()[1].reshape(3, -1)[2]
    assert np.allclose(uz, u0 / (1 + k * u0 * n), rtol=1e-3)


def _vdw_state(p, P, h, guess):
    # (rho, T) with pressure P and specific enthalpy h = e + P/rho
    from scipy import optimize
    L = orc.lib()

    def res(x):
        rho, T = x
        Pc = L.orc_eos_P(p, rho, T)
        return [Pc / P - 1.0, (L.orc_eos_e(p, rho, T) + Pc / rho) / h - 1.0]

    return optimize.fsolve(res, guess, xtol=1e-13)


@pytest.mark.parametrize("Pr,hr", [(15.0, 5.0), (3.0, 11.25)])
def test_throttling_reproduces_the_joule_thomson_coefficient(Pr, hr):
    # Throttling (Sec. III.B): a Darcy throttle F = -K phi rho u with Q = -F.u between an inlet at fixed
    # (P_in, T_in) and an outlet at 0.98 P_in keeps h uniform, and Delta T / Delta P is the Joule-Thomson
    # coefficient mu_JT = -(1/c_P) [1/rho - T P_T / (rho^2 P_rho)] of van der Waals (both signs: the
    # states lie on either side of the inversion line).  Reduced fluid b = 2/21, Tc, Pc scaled down so
    # that the dense states' sound speed stays near 0.3 lattice speeds; low conduction (k/mu = 0.35).
    a, b, cv = wl.VDW_A * 0.05, wl.VDW_B, 2.5
    Tc, Pc = 8 * a / (27 * b), a / (27 * b * b)
    p = orc.make_params(dim=3, nx=1, ny=1, nz=40, eos="vdw", R=1.0, cv=cv, a=a, b=b)
    P_in = Pr * Pc
    rho_in, T_in = _vdw_state(p, P_in, hr * Tc, [2.0 / (3.0 * b), 1.5 * Tc])
    c = wl.Case(name="throttle", dim=3, nx=1, ny=1, nz=40, zwalls=2, eos="vdw", R=1.0, cv=cv, a=a, b=b,
                k_over_mu=0.35, eta_over_mu=3.0, tau_f=2.0, tau_g=2.0, phi_central=1, face_kind=(5, 3),
                face_P=(P_in, 0.98 * P_in), Tw_lo=T_in, Tw_hi=T_in, throttle_K=0.02, throttle_sigma=3.0,
                init=dict(kind="duct", rho0=rho_in, u0=0.0, T0=T_in))
    threads = orc.get_threads()
    orc.set_threads(1)
    try:
        o = run_oracle(c, 25000)
    finally:
        orc.set_threads(threads)
    rho, u, T = o.moments()
    uz = u.reshape(3, -1)[2]
    L = orc.lib()
    P = np.array([L.orc_eos_P(o.p, r, t) for r, t in zip(rho, T)])
    h = np.array([L.orc_eos_e(o.p, r, t) for r, t in zip(rho, T)]) + P / rho
    assert np.ptp((rho * uz)[1:-1]) <= 1e-6 * (rho * uz).mean()
    assert np.ptp(h + 0.5 * uz ** 2) <= 2e-3 * abs(h.mean())
    r_m, T_m = 0.5 * (rho[1] + rho[-2]), 0.5 * (T[1] + T[-2])
    P_rho, P_T = L.orc_eos_dPdrho(o.p, r_m, T_m), L.orc_eos_dPdT(o.p, r_m, T_m)
    c_P = L.orc_eos_cv(o.p, r_m, T_m) + T_m * P_T ** 2 / (r_m ** 2 * P_rho)
    mu_jt = -(1.0 / r_m - T_m * P_T / (r_m ** 2 * P_rho)) / c_P
    dTdP = (T[-2] - T[1]) / (P[-2] - P[1])
    assert dTdP == pytest.approx(mu_jt, rel=0.02)


def test_bench_recipes_of_the_wall_and_duct_forms_are_sound():
    # the thermal Couette and Fanno duct workloads the benchmark times, at reduced size: finite fields,
    # the wall temperatures held, a uniform mass flux along the ducts after the inlet transient
    tc = wl.thermal_couette(6, 12)
    o = run_oracle(tc, 300)
    rho, u, T = o.moments()
    plane = tc.nx * tc.ny
    assert np.all(np.isfinite(rho)) and np.all(rho > 0)
    assert np.all(T[:plane] == tc.Tw_lo) and np.all(T[-plane:] == tc.Tw_hi)
    fd = wl.fanno_duct(2, 40)
    o = run_oracle(fd, 4000)
    rho, u, T = o.moments()
    uz = u.reshape(3, -1)[2].reshape(fd.nz, -1)
    m = (rho.reshape(fd.nz, -1) * uz).mean(axis=1)
    assert np.all(np.isfinite(m)) and m.min() > 0
    assert np.ptp(m[1:-1]) <= 1e-3 * m.mean()


# Supersonic inlet (Sec. III.A: Rayleigh and Fanno flow entering at Ma 1.5): static inlet
# (P, T, u given), extrapolated outlet, the upwind-biased Phi.  Uniform supersonic flow of
# this step is linearly stable only at low lattice temperature and tau >= 1 (see
# test_oracle_stability); T_in = 0.02, tau = 1.
SS_T, SS_MA, SS_TAU = 0.02, 1.5, 1.0
SS_U = SS_MA * math.sqrt(GAM * R_GAS * SS_T)


def _ss_duct(nz, q=0.0, friction=0.0):
    return wl.Case(name="ss_duct", dim=3, nx=1, ny=1, nz=nz, zwalls=2, eos="ideal", R=R_GAS, cv=CV,
                   k_over_mu=CP / 0.71, tau_f=SS_TAU, tau_g=SS_TAU, phi_central=0, q=q, zlo=0, zhi=0,
                   friction=friction, face_kind=(2, 4), face_P=(SS_T, 0.0), uw_lo=(0.0, 0.0, SS_U),
                   Tw_lo=SS_T, Tw_hi=SS_T, init=dict(kind="duct", rho0=1.0, u0=SS_U, T0=SS_T))


def test_supersonic_rayleigh_flow_relations():
    # heat addition decelerates a supersonic flow towards Ma 1 along one Rayleigh line
    nz, q = 50, 8e-7
    rho, uz, T, P, Ma = _profiles(_ss_duct(nz, q=q), 20000)
    mdot = rho * uz
    assert np.ptp(mdot[1:-1]) <= 1e-7 * mdot.mean()
    assert 1.0 < Ma[-2] < Ma[1] - 1e-3
    Ts = T * (1 + GAM * Ma ** 2) ** 2 / ((1 + GAM) ** 2 * Ma ** 2)
    Ps = P * (1 + GAM * Ma ** 2) / (1 + GAM)
    assert np.ptp(Ts[1:-1]) <= 1e-4 * Ts.mean()
    assert np.ptp(Ps[1:-1]) <= 1e-4 * Ps.mean()
    H = CP * T + 0.5 * uz ** 2
    Hana = H[1] + q * (np.arange(nz) - 1) / mdot.mean()
    assert np.max(np.abs(H - Hana)[1:-1]) <= 0.03 * q * nz / mdot.mean()


def test_supersonic_fanno_flow_relations():
    # friction decelerates a supersonic flow towards Ma 1 along one Fanno line (duct well
    # inside the choking length 4 f L*/D = 0.136 at Ma 1.5), total enthalpy constant
    nz = 50
    rho, uz, T, P, Ma = _profiles(_ss_duct(nz, friction=5e-4), 20000)
    assert np.ptp((rho * uz)[1:-1]) <= 1e-7 * (rho * uz).mean()
    assert 1.0 < Ma[-2] < Ma[1] - 0.05
    Ts = T * (2 + (GAM - 1) * Ma ** 2) / (1 + GAM)
    Ps = P * Ma * np.sqrt((2 + (GAM - 1) * Ma ** 2) / (1 + GAM))
    assert np.ptp(Ts[1:-1]) <= 1e-3 * Ts.mean()
    assert np.ptp(Ps[1:-1]) <= 2e-3 * Ps.mean()
    H = CP * T + 0.5 * uz ** 2
    assert np.ptp(H[1:-1]) <= 1e-3 * H.mean()
