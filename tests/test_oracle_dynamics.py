"""Pins of the oracle's full time step against what the paper and the
mathematics fix: exact mass conservation, the discrete momentum and energy
budgets of the half-force moments (Eqs. def_u, def_E), uniform acceleration and
isochoric heating in closed form, the hydrodynamic-limit decay rates
(Sec. II.D), bounce-back walls, and van der Waals liquid-vapour coexistence at
the Maxwell densities (Sec. III.B)."""
import math

import numpy as np
import pytest
from scipy import optimize

from oracle import oracle as orc
from paper_2609_28679_b300 import workloads as wl
from tests.util import oracle_params, run_oracle, maxwell


def _uniform_case(eos="ideal", dim=2, n=4, **kw):
    init = dict(kind="uniform", rho0=kw.pop("rho0", 1.0), T0=kw.pop("T0", 0.3))
    return wl.Case(name="uniform", dim=dim, nx=n, ny=n, nz=n if dim == 3 else 1, eos=eos, init=init, **kw)


def test_mass_is_conserved_exactly():
    c = wl.vdw_spinodal(n=16, steps=0)
    o = run_oracle(c, 0)
    m0 = o.invariants()[0]
    o.step(200)
    assert abs(o.invariants()[0] - m0) <= 1e-13 * m0


@pytest.mark.parametrize("case_fn", ["vdw", "ideal3d", "pr3d_walls"])
def test_momentum_and_energy_budgets(case_fn):
    # M(n) = sum(rho u), En(n) = sum(rho E) with the half-force moments; then
    # M(n+1) - M(n) = (SF(n) + SF(n+1))/2 and En(n+1) - En(n) = (SS(n) + SS(n+1))/2, S = u.F + Q.
    if case_fn == "vdw":
        c = wl.vdw_spinodal(n=16, steps=0)
        c.q = 3e-5
        c.accel = (2e-5, -1e-5, 0.0)
        exact_energy, walls = True, False
    elif case_fn == "ideal3d":
        c = wl.acoustic_shear(n=8, steps=0)
        c = wl.Case(**{**c.__dict__, "dim": 3, "nz": 8, "accel": (1e-5, 2e-5, -1e-5)})
        exact_energy, walls = True, False
    else:
        c = wl.pr_heated_slab(n=6, nz=8, steps=0)
        exact_energy, walls = False, True
    D = c.dim
    o = run_oracle(c, 0)
    prev = o.invariants()
    for _ in range(30):
        o.step(1)
        cur = o.invariants()
        M0, M1 = prev[1:1 + D], cur[1:1 + D]
        F0, F1 = prev[D + 2:2 * D + 2], cur[D + 2:2 * D + 2]
        budget = M1 - M0 - 0.5 * (F0 + F1)
        if not walls:  # no-slip walls take up momentum in every component
            # rounding of N per-cell terms of size ~ rho |u|, |F|
            assert np.max(np.abs(budget)) <= 1e-13 * cur[0]
        dE = cur[1 + D] - prev[1 + D] - 0.5 * (prev[-1] + cur[-1])
        if exact_energy:
            assert abs(dE) <= 1e-12 * abs(cur[1 + D])
        else:
            # Peng-Robinson: c_v depends on T, so e(T*) - e(T) differs from c_v (T* - T) at second order
            assert abs(dE) <= 1e-6 * abs(prev[-1]) + 1e-12 * abs(cur[1 + D])
        prev = cur


def test_uniform_acceleration_is_galilean():
    # Uniform state, F = rho a: u(n) = (n + 1/2) a exactly and e stays constant (no heating):
    # the -F.F/(2 rho^2 c_v) term of Eq. sh_T_1 balances the kinetic energy of u*.
    c = _uniform_case(eos="vdw", rho0=2.0, T0=0.6, a=9 / 49, b=2 / 21, accel=(3e-3, -2e-3, 0.0))
    c.phi_central = 0  # upwind-biased Phi with a nonzero uniform u
    o = run_oracle(c, 0)
    _, _, T0 = o.moments()
    n = 40
    o.step(n)
    rho, u, T = o.moments()
    np.testing.assert_allclose(u[0], (n + 0.5) * 3e-3, rtol=1e-12)
    np.testing.assert_allclose(u[1], -(n + 0.5) * 2e-3, rtol=1e-12)
    np.testing.assert_allclose(T, T0, rtol=1e-12)


@pytest.mark.parametrize("eos", ["ideal", "vdw"])
def test_isochoric_heating(eos):
    # Uniform Q on a periodic box at rest: T(n) = T0 + (n + 1/2) Q/(rho c_v) for constant c_v
    # (the isochoric-heating step of the Joule-Thomson measurement, Sec. III.B).
    kw = dict(a=9 / 49, b=2 / 21) if eos == "vdw" else {}
    rho0, T0, Q = 2.0, 0.6, 1e-4
    c = _uniform_case(eos=eos, rho0=rho0, T0=T0, q=Q, **kw)
    o = run_oracle(c, 0)
    n = 100
    o.step(n)
    rho, u, T = o.moments()
    np.testing.assert_allclose(T, T0 + (n + 0.5) * Q / (rho0 * 2.5), rtol=1e-12)
    np.testing.assert_allclose(rho, rho0, rtol=1e-14)
    assert np.max(np.abs(u)) < 1e-14


def _mode_amplitude(field, nx):
    # |Fourier coefficient| of the k = 2 pi / nx mode along x (field is uniform in y)
    prof = field.reshape(-1, nx).mean(axis=0)
    x = np.arange(nx)
    return 2.0 / nx * np.abs(np.sum(prof * np.exp(-2j * math.pi * x / nx)))


def test_shear_wave_decay_rate():
    # Linearised NSF (Sec. II.D): u_y(k,t) ~ exp(-nu k^2 t) with nu = mu/rho = tau theta.
    nx, tau, T0 = 48, 0.8, 0.3
    c = wl.Case(name="shear", dim=2, nx=nx, ny=1, eos="ideal", R=1.0, cv=2.5, k_over_mu=3.5 / 0.71,
                tau_f=tau, tau_g=tau, init=dict(kind="waves", rho0=1.0, amp_rho=0.0, amp_u=1e-4, T0=T0))
    o = run_oracle(c, 0)
    amps, ts = [], [50, 150, 250, 350]
    t = 0
    for tt in ts:
        o.step(tt - t)
        t = tt
        amps.append(_mode_amplitude(o.moments()[1][1], nx))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    k = 2 * math.pi / nx
    assert rate == pytest.approx(tau * T0 * k * k, rel=0.01)


def test_shear_wave_decay_rate_constant_mu():
    # The paper's own parameterisation tau = mu / P per cell (Sec. II.C): the kinematic viscosity is
    # nu = mu / rho, here at rho0 = 2 so that a tau taken as mu itself (nu = mu theta) would fail.
    nx, mu, rho0, T0 = 48, 0.48, 2.0, 0.3
    c = wl.Case(name="shear_mu", dim=2, nx=nx, ny=1, eos="ideal", R=1.0, cv=2.5, k_over_mu=3.5 / 0.71,
                mu=mu, init=dict(kind="waves", rho0=rho0, amp_rho=0.0, amp_u=1e-4, T0=T0))
    o = run_oracle(c, 0)
    amps, ts = [], [50, 150, 250, 350]
    t = 0
    for tt in ts:
        o.step(tt - t)
        t = tt
        amps.append(_mode_amplitude(o.moments()[1][1], nx))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    k = 2 * math.pi / nx
    assert rate == pytest.approx(mu / rho0 * k * k, rel=0.01)


def test_constant_mu_equals_constant_tau_at_uniform_pressure():
    # With P uniform and constant in time (a state at rest), tau = mu / P is the constant mu / P0,
    # so both parameterisations take the same steps (to rounding of beta).
    base = dict(dim=2, nx=6, ny=5, eos="vdw", R=1.0, cv=2.5, a=9 / 49, b=2 / 21, k_over_mu=3.5,
                init=dict(kind="uniform", rho0=1.3, T0=0.8))
    ca = wl.Case(name="tau", tau_f=0.7, tau_g=0.7, **base)
    oa = run_oracle(ca, 0)
    P0 = orc.EoS(orc.params_from_case(ca)).P(1.3, 0.8)
    cb = wl.Case(name="mu", mu=0.7 * P0, **base)
    ob = run_oracle(cb, 0)
    oa.step(30)
    ob.step(30)
    fa, ga = oa.populations()
    fb, gb = ob.populations()
    assert np.max(np.abs(fa - fb)) <= 1e-14 and np.max(np.abs(ga - gb)) <= 1e-14


def test_sound_speed_and_acoustic_damping():
    # Uniform-T density pulse: the acoustic part oscillates at c_s k with c_s^2 = gamma R T (ideal gas)
    # and decays at Gamma = k^2/2 [2(D-1)/D nu + (gamma - 1) chi] (eta = 0), chi = k_cond/(rho c_p).
    nx, tau, T0 = 48, 0.8, 0.3
    c = wl.Case(name="sound", dim=2, nx=nx, ny=1, eos="ideal", R=1.0, cv=2.5, k_over_mu=3.5 / 0.71,
                tau_f=tau, tau_g=tau, init=dict(kind="waves", rho0=1.0, amp_rho=1e-4, amp_u=0.0, T0=T0))
    o = run_oracle(c, 0)
    x = np.arange(nx)
    ts, sig = np.arange(0, 400), []
    for t in ts:
        rho = o.moments()[0]
        sig.append(2.0 / nx * np.sum((rho - rho.mean()) * np.sin(2 * math.pi * x / nx)))
        o.step(1)
    sig = np.array(sig)
    k, gam = 2 * math.pi / nx, 1.4
    nu = tau * T0
    chi = (3.5 / 0.71) * tau * T0 / 3.5  # k_cond/(rho c_p) with mu = tau P, rho = 1
    cs = math.sqrt(gam * T0)
    Gam = 0.5 * k * k * (2 * (2 - 1) / 2 * nu + (gam - 1) * chi)
    Dt = 0.5 * k * k * 0  # placeholder, the entropy mode is fitted as a free exponential

    def model(t, A, w, G, B, lam):
        return A * np.cos(w * t) * np.exp(-G * t) + B * np.exp(-lam * t)

    p0 = [1e-4 / gam, cs * k, Gam, 1e-4 * (1 - 1 / gam), chi * k * k]
    popt, _ = optimize.curve_fit(model, ts, sig, p0=p0, maxfev=20000)
    assert popt[1] == pytest.approx(cs * k, rel=0.01)
    assert popt[2] == pytest.approx(Gam, rel=0.1)
    assert popt[4] == pytest.approx(chi * k * k, rel=0.1)


def test_bounce_back_walls_conserve_mass_and_energy():
    # Half-way bounce-back (Sec. III.A) on z: mass exact; energy follows the budget with Q.
    c = wl.Case(name="walls", dim=3, nx=4, ny=3, nz=10, zwalls=1, eos="vdw", R=1.0, cv=2.5, a=9 / 49,
                b=2 / 21, kappa=0.1, k_over_mu=3.5, accel=(1e-4, 0.0, -3e-4), q=2e-5, zlo=0, zhi=3,
                init=dict(kind="noisy_temperature", rho0=1.2, amp=0.05, T0=0.6, seed=9))
    o = run_oracle(c, 0)
    prev = o.invariants()
    for _ in range(20):
        o.step(1)
        cur = o.invariants()
        assert abs(cur[0] - prev[0]) <= 1e-14 * cur[0]
        dE = cur[4] - prev[4] - 0.5 * (prev[-1] + cur[-1])
        assert abs(dE) <= 1e-12 * abs(cur[4])
        prev = cur


def test_poiseuille_between_bounce_back_walls():
    # Force-driven flow between half-way bounce-back walls at z = -1/2 and nz - 1/2:
    # u_x(z) = a/(2 nu) (z + 1/2)(nz - 1/2 - z), nu = tau theta (Sec. III.A, Poiseuille).
    # The curvature pins the viscosity; half-way bounce-back with BGK adds a uniform slip of
    # second order in the grid spacing, so the offset is only bounded.
    nz, a, tau, T0 = 16, 1e-6, 0.8, 0.3
    c = wl.Case(name="pois", dim=3, nx=1, ny=1, nz=nz, zwalls=1, eos="ideal", R=1.0, cv=2.5,
                k_over_mu=3.5 / 0.71, tau_f=tau, tau_g=tau, accel=(a, 0.0, 0.0),
                init=dict(kind="uniform", rho0=1.0, T0=T0))
    o = run_oracle(c, 6000)
    rho, u, T = o.moments()
    z = np.arange(nz)
    nu = tau * T0
    shape = (z + 0.5) * (nz - 0.5 - z)
    A, B = np.polyfit(shape, u[0], 1)
    assert A == pytest.approx(a / (2 * nu), rel=0.01)
    assert abs(B) <= 0.05 * A * shape.max()
    assert np.max(np.abs(u[0] - (A * shape + B))) <= 1e-3 * A * shape.max()


def test_poiseuille_constant_mu():
    # Poiseuille curvature a / (2 nu) with nu = mu / rho for tau = mu / P per cell (Sec. II.C, III.A).
    nz, a, mu, rho0, T0 = 16, 1e-6, 0.36, 1.5, 0.3
    c = wl.Case(name="pois_mu", dim=3, nx=1, ny=1, nz=nz, zwalls=1, eos="ideal", R=1.0, cv=2.5,
                k_over_mu=3.5 / 0.71, mu=mu, accel=(a, 0.0, 0.0), init=dict(kind="uniform", rho0=rho0, T0=T0))
    o = run_oracle(c, 6000)
    rho, u, T = o.moments()
    z = np.arange(nz)
    shape = (z + 0.5) * (nz - 0.5 - z)
    A, B = np.polyfit(shape, u[0], 1)
    assert A == pytest.approx(a / (2 * mu / rho0), rel=0.01)


def test_isothermal_poiseuille():
    # Isothermal mode (Sec. III.A: the g equation is not solved): force-driven flow between half-way
    # bounce-back walls keeps the curvature a / (2 nu), nu = tau theta, and the temperature stays put.
    nz, a, tau, T0 = 16, 1e-6, 0.8, 0.3
    c = wl.Case(name="pois_iso", dim=3, nx=1, ny=1, nz=nz, zwalls=1, eos="ideal", R=1.0, cv=2.5,
                k_over_mu=3.5 / 0.71, tau_f=tau, tau_g=tau, accel=(a, 0.0, 0.0), isothermal=1,
                init=dict(kind="uniform", rho0=1.0, T0=T0))
    o = run_oracle(c, 6000)
    rho, u, T = o.moments()
    z = np.arange(nz)
    shape = (z + 0.5) * (nz - 0.5 - z)
    A, B = np.polyfit(shape, u[0], 1)
    assert A == pytest.approx(a / (2 * tau * T0), rel=0.01)
    assert np.all(T == T0)


def _womersley(xi, t, g, omega, Wo):
    # Womersley's pulsatile channel flow driven by a cos(omega t) (Sec. III.A), xi = x / L in [0, 1]
    si = np.sqrt(1j)
    prof = 1.0 - np.cosh(si * Wo * (xi - 0.5)) / np.cosh(si * Wo / 2.0)
    return np.real(g / (1j * omega) * prof * np.exp(1j * omega * t))


def test_isothermal_womersley():
    # Isothermal pulsatile flow between half-way bounce-back walls at z = -1/2 and nz - 1/2 (L = nz),
    # body acceleration g cos(omega t) set before every step, started from the analytic profile
    # at t = 0 and compared one period later with nu = tau theta.
    nz, tau, T0, g, Wo = 32, 0.8, 0.3, 1e-6, 4.0
    nu = tau * T0
    omega = Wo * Wo * nu / (nz * nz)
    period = int(round(2 * math.pi / omega))
    omega = 2 * math.pi / period
    Wo = nz * math.sqrt(omega / nu)
    xi = (np.arange(nz) + 0.5) / nz
    c = wl.Case(name="womersley", dim=3, nx=1, ny=1, nz=nz, zwalls=1, eos="ideal", R=1.0, cv=2.5,
                k_over_mu=3.5 / 0.71, tau_f=tau, tau_g=tau, isothermal=1, init=dict(kind="uniform", rho0=1.0, T0=T0))
    u0 = np.zeros((3, nz))
    u0[0] = _womersley(xi, 0.0, g, omega, Wo)
    o = orc.Oracle(oracle_params(c))
    o.init(np.ones(nz), u0, np.full(nz, T0))
    for n in range(period):
        o.set_accel((g * math.cos(omega * n), 0.0, 0.0))
        o.step(1)
        if n + 1 in (period // 4, period // 2, period):
            ux = o.moments()[1][0]
            ref = _womersley(xi, n + 1, g, omega, Wo)
            err = np.sqrt(np.sum((ux - ref) ** 2) / np.sum(ref ** 2))
            assert err <= 0.01, (n + 1, err)


def test_isothermal_sound_speed():
    # Without the energy equation a density wave travels at the isothermal sound speed
    # c_T = sqrt((dP/drho)_T) = sqrt(R T) of the ideal gas, not the adiabatic sqrt(gamma R T).
    nx, tau, T0 = 48, 0.8, 0.3
    c = wl.Case(name="sound_iso", dim=2, nx=nx, ny=1, eos="ideal", R=1.0, cv=2.5, k_over_mu=3.5 / 0.71,
                tau_f=tau, tau_g=tau, isothermal=1,
                init=dict(kind="waves", rho0=1.0, amp_rho=1e-4, amp_u=0.0, T0=T0))
    o = run_oracle(c, 0)
    x = np.arange(nx)
    ts, sig = np.arange(0, 300), []
    for t in ts:
        rho = o.moments()[0]
        sig.append(2.0 / nx * np.sum((rho - rho.mean()) * np.sin(2 * math.pi * x / nx)))
        o.step(1)
    sig = np.array(sig)
    k = 2 * math.pi / nx

    def model(t, A, w, G):
        return A * np.cos(w * t) * np.exp(-G * t)

    popt, _ = optimize.curve_fit(model, ts, sig, p0=[1e-4, math.sqrt(T0) * k, 1e-3], maxfev=20000)
    assert popt[1] == pytest.approx(math.sqrt(T0) * k, rel=0.01)


def _maxwell(eos, T):
    return maxwell(eos, T)


def test_maxwell_construction_reproduces_textbook_vdw():
    # Reduced vdW coexistence at Tr = 0.9 (textbook): rho_v/rho_c ~ 0.4257, rho_l/rho_c ~ 1.6573.
    eos = orc.EoS(orc.make_params(eos="vdw", R=1.0, cv=2.5, a=9 / 49, b=2 / 21))
    rv, rl = _maxwell(eos, 0.9 * 4 / 7)
    assert rv / 3.5 == pytest.approx(0.4257, abs=2e-3)
    assert rl / 3.5 == pytest.approx(1.6573, abs=2e-3)


@pytest.mark.slow
def test_vdw_coexistence_densities():
    # Liquid column in a periodic 1-D box with the Korteweg force (Sec. III.B): the bulk densities
    # relax to the Maxwell densities at the (measured) temperature.
    nx = 160
    eos = orc.EoS(orc.make_params(eos="vdw", R=1.0, cv=2.5, a=wl.VDW_A, b=wl.VDW_B))
    T0 = 0.9 * wl.VDW_TC
    rv, rl = _maxwell(eos, T0)
    x = np.arange(nx)
    prof = rv + (rl - rv) * 0.5 * (np.tanh((x - nx / 4) / 2.5) - np.tanh((x - 3 * nx / 4) / 2.5))
    c = wl.Case(name="coex", dim=2, nx=nx, ny=1, eos="vdw", R=1.0, cv=2.5, a=wl.VDW_A, b=wl.VDW_B,
                kappa=wl.VDW_KAPPA, eta_over_mu=wl.VDW_ETA, k_over_mu=3.5, phi_central=1,
                init=dict(kind="uniform"))
    o = orc.Oracle(oracle_params(c))
    o.init(prof, np.zeros((2, nx)), np.full(nx, T0))
    o.step(6000)
    rho, u, T = o.moments()
    rv_T, rl_T = _maxwell(eos, float(T.mean()))
    assert rho[nx // 2] == pytest.approx(rl_T, rel=0.02)
    assert rho[0] == pytest.approx(rv_T, rel=0.02)
    assert np.max(np.abs(u)) < 1e-3


def test_per_cell_heat_field_equals_the_uniform_source():
    # Q(x) given per cell (Eq. force_decomposition's generic source) adds to the uniform Q: a field equal
    # to q everywhere reproduces q bit for bit
    c = wl.acoustic_shear(n=12, storage="f64")
    a = run_oracle(c, 0)
    q = c.q
    c0 = wl.acoustic_shear(n=12, storage="f64")
    c0.q = 0.0
    b = run_oracle(c0, 0)
    b.set_fields(None, np.full(c0.ncell, q))
    a.step(15)
    b.step(15)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_per_cell_force_field_follows_the_momentum_budget():
    # F_B(x) per cell: total momentum changes by the total force each step (half-force moments, Eq. def_u)
    c = wl.vdw_spinodal(n=10, storage="f64")
    c.accel = (0.0, 0.0, 0.0)
    o = run_oracle(c, 0)
    rng = np.random.default_rng(3)
    F = 1e-5 * rng.standard_normal((2, c.ncell))
    o.set_fields(F, None)
    prev = o.invariants()
    for _ in range(10):
        o.step(1)
        cur = o.invariants()
        for a in range(2):
            assert cur[1 + a] - prev[1 + a] == pytest.approx(0.5 * (prev[4 + a] + cur[4 + a]), rel=1e-9, abs=1e-15)
        prev = cur
    # the Korteweg force sums to zero on a periodic grid; what is left is the field's total
    assert cur[4] == pytest.approx(F[0].sum(), rel=1e-9, abs=1e-14)
