"""Duct ends and duct friction (the 1-D duct flows of Sec. III.A, run as
columns of D3Q27) on the GPU split kernels, through the C ABI, against the
FP64 CPU oracle on the same seeded inputs: populations and moments element by
element for every face kind and for friction (also in 2-D), the conservation
totals, the steady Rayleigh relations, and the API rules.

Tolerances as in the other parity tests: float64 1e-12 relative (u to 1e-12 of
max(max|u_ref|, 1e-3)), float32 1e-5 (u to 1e-5 of the lattice speed)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_28679_b300 import lbm
from paper_2609_28679_b300 import workloads as wl
from tests.util import oracle_params, rel_linf

pytestmark = pytest.mark.gpu

R_GAS, CV = 1.0, 2.5
CP, GAM = R_GAS + CV, (R_GAS + CV) / CV
T_IN, P_IN, MA_IN = 0.1, 0.1, 0.3
T0 = T_IN * (1.0 + 0.5 * (GAM - 1.0) * MA_IN ** 2)
P0 = P_IN * (T0 / T_IN) ** (CP / R_GAS)
U_IN = MA_IN * math.sqrt(GAM * R_GAS * T_IN)


def _duct(nz=40, nx=1, ny=1, q=0.0, friction=0.0, kinds=(1, 3), face_P=(P0, 0.08), uw_lo=(0.0, 0.0, 0.0),
          T_lo=T0, storage="f64", amp=0.0):
    init = dict(kind="duct", rho0=P_IN / (R_GAS * T_IN), u0=U_IN, T0=T_IN)
    c = wl.Case(name="duct", dim=3, nx=nx, ny=ny, nz=nz, zwalls=2, eos="ideal", R=R_GAS, cv=CV,
                k_over_mu=CP / 0.71, tau_f=0.8, tau_g=0.8, phi_central=1, q=q, zlo=0, zhi=0, friction=friction,
                face_kind=kinds, face_P=face_P, uw_lo=uw_lo, Tw_lo=T_lo, Tw_hi=T_lo, storage=storage, init=init)
    return c


def _noisy_fields(c, amp, seed):
    rho, u, T = c.fields()
    rho = rho * (1.0 + amp * wl.uniform_pm1(seed, c.ncell))
    T = T * (1.0 + amp * wl.uniform_pm1(seed + 1, c.ncell))
    return rho, u, T


SPLIT, ZMARCH = lbm.LBM_KERNEL_SPLIT, lbm.LBM_KERNEL_ZMARCH


def _pair(c, steps, fields, variant=SPLIT):
    sim = lbm.Simulation(c)
    tile = (0, 0, 0)
    if isinstance(variant, tuple):
        variant, tile = variant
    lbm.lbm_set_kernel(sim.h, variant, *tile)
    assert sim.kernel()[0] == variant
    sim.init(fields)
    sim.step(steps)
    o = orc.Oracle(oracle_params(c))
    o.init(*fields)
    o.step(steps)
    return sim, o


def _compare(sim, o, tol, f32=False):
    f, g = sim.populations()
    fr, gr = o.populations()
    assert rel_linf(f, fr.ravel()) <= tol
    assert rel_linf(g, gr.ravel()) <= tol
    rho, u, T = sim.moments()
    rr, ur, Tr = o.moments()
    assert rel_linf(rho, rr) <= tol
    assert rel_linf(T, Tr) <= tol
    tol_u = tol if f32 else tol * max(float(np.max(np.abs(ur))), 1e-3)
    assert float(np.max(np.abs(u - ur.ravel()))) <= tol_u


@pytest.mark.parametrize("kinds,face_P,uw_lo,T_lo", [
    ((1, 3), (P0, 0.08), (0.0, 0.0, 0.0), T0),          # subsonic: total inlet, pressure outlet
    ((2, 4), (P_IN, 0.0), (0.0, 0.0, U_IN), T_IN),      # static inlet, extrapolated outlet
    ((2, 3), (P_IN, 0.09), (0.0, 0.0, U_IN), T_IN),
])
@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2)])
@pytest.mark.parametrize("variant", [SPLIT, (ZMARCH, (30, 6, 4))])
def test_f64_duct_ends_match_oracle(kinds, face_P, uw_lo, T_lo, nx, ny, variant):
    c = _duct(nz=40, nx=nx, ny=ny, q=4e-5, kinds=kinds, face_P=face_P, uw_lo=uw_lo, T_lo=T_lo)
    sim, o = _pair(c, 120, _noisy_fields(c, 0.01, 31), variant)
    _compare(sim, o, 1e-12)


@pytest.mark.parametrize("variant", [SPLIT, (ZMARCH, (30, 14, 32)), (ZMARCH, (30, 6, 4))])
def test_f64_fanno_friction_matches_oracle(variant):
    c = _duct(nz=40, friction=4e-3)
    sim, o = _pair(c, 150, _noisy_fields(c, 0.01, 32), variant)
    _compare(sim, o, 1e-12)


def test_f64_friction_2d_periodic_matches_oracle_and_conserves_energy():
    # friction in a periodic 2-D van der Waals flow: parity, and Q = -F.u keeps total energy exact
    # (friction the only force, so that sum (u.F + Q) vanishes)
    c = wl.vdw_spinodal(n=24, storage="f64")
    c.friction, c.accel, c.kappa = 0.05, (0.0, 0.0, 0.0), 0.0
    c.init = dict(kind="waves", rho0=wl.VDW_RHO_MID_090, amp_rho=0.01, amp_u=0.05, T0=0.1)
    fields = c.fields()
    fields[1][0] += 0.04  # mean flow along x
    sim, o = _pair(c, 30, fields)
    _compare(sim, o, 1e-12)
    gi = sim.invariants()[0]
    oi = o.invariants()
    assert np.all(np.abs(gi - oi) <= 1e-12 * np.maximum(np.abs(oi), np.abs(oi[0])))
    assert abs(gi[-1]) <= 1e-12 * abs(gi[3])  # sum (u.F + Q) = 0


@pytest.mark.parametrize("variant", [SPLIT, (ZMARCH, (30, 6, 4))])
def test_f32_duct_matches_oracle(variant):
    c = _duct(nz=40, q=4e-5, friction=2e-3, storage="f32")
    sim, o = _pair(c, 120, _noisy_fields(c, 0.01, 33), variant)
    _compare(sim, o, 1e-5, f32=True)


def test_rayleigh_relations_on_the_gpu():
    nz, q = 50, 4e-5
    c = _duct(nz=nz, q=q)
    sim = lbm.Simulation(c)
    sim.init()
    sim.step(20000)
    rho, u, T = sim.moments()
    uz = u.reshape(3, -1)[2]
    P = rho * R_GAS * T
    Ma = uz / np.sqrt(GAM * R_GAS * T)
    assert np.ptp((rho * uz)[1:-1]) <= 1e-10 * (rho * uz).mean()
    Ts = T * (1 + GAM * Ma ** 2) ** 2 / ((1 + GAM) ** 2 * Ma ** 2)
    Ps = P * (1 + GAM * Ma ** 2) / (1 + GAM)
    assert np.ptp(Ts[1:-1]) <= 1e-3 * Ts.mean()
    assert np.ptp(Ps[1:-1]) <= 1e-3 * Ps.mean()


def test_duct_api_rules():
    c = _duct(nz=12, friction=1e-3)
    lat, eos, force, heat = lbm.structs_from_case(c)
    h = lbm.lbm_create(lat, eos, c.tau_f, c.tau_g, force, heat)
    try:
        assert lbm.lbm_get_kernel(h)[0] == lbm.LBM_KERNEL_ZMARCH  # extrapolated faces: the z-march
        rho, u, T = c.fields()
        lbm.lbm_init(h, rho, u.ravel(), T, 0)
        lbm.lbm_set_face(h, 0, lbm.LBM_FACE_INLET_TOTAL, None, T0, P0)
        with pytest.raises(lbm.LbmError, match="every face"):
            lbm.lbm_step(h, 1)  # face 1 not set yet
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_face(h, 1, lbm.LBM_FACE_OUTLET_P, None, 0.0, -1.0)
        lbm.lbm_set_face(h, 1, lbm.LBM_FACE_OUTLET_P, None, 0.0, 0.08)
        lbm.lbm_step(h, 2)
        with pytest.raises(lbm.LbmError, match="split"):
            lbm.lbm_set_kernel(h, lbm.LBM_KERNEL_FUSED)
    finally:
        lbm.lbm_destroy(h)
    # friction without extrapolated faces runs on the split kernels only (2-D, and 3-D periodic)
    p = wl.vdw_spinodal(n=16, storage="f64")
    p.friction = 1e-3
    sim = lbm.Simulation(p)
    assert sim.kernel()[0] == lbm.LBM_KERNEL_SPLIT
    sim.close()
    p3 = wl.pr_heated_slab(n=8, nz=6, storage="f64")
    p3.friction = 1e-3
    sim = lbm.Simulation(p3)
    assert sim.kernel()[0] == lbm.LBM_KERNEL_SPLIT
    with pytest.raises(lbm.LbmError, match="split"):
        lbm.lbm_set_kernel(sim.h, lbm.LBM_KERNEL_ZMARCH)
    sim.close()
    # a total-state inlet needs the ideal gas
    v = _duct(nz=12)
    v.eos, v.a, v.b = "vdw", wl.VDW_A, wl.VDW_B
    v.face_kind = (0, 0)
    sim = lbm.Simulation(v)
    with pytest.raises(lbm.LbmError, match="ideal"):
        lbm.lbm_set_face(sim.h, 0, lbm.LBM_FACE_INLET_TOTAL, None, 0.1, 0.1)
    sim.close()


def _throttle_case(storage="f64", Pr=15.0, hr=5.0):
    from scipy import optimize

    a, b, cv = wl.VDW_A * 0.05, wl.VDW_B, 2.5
    Tc, Pc = 8 * a / (27 * b), a / (27 * b * b)
    p = orc.make_params(dim=3, nx=1, ny=1, nz=40, eos="vdw", R=1.0, cv=cv, a=a, b=b)
    L = orc.lib()
    P_in, h_in = Pr * Pc, hr * Tc

    def res(x):
        P = L.orc_eos_P(p, x[0], x[1])
        return [P / P_in - 1.0, (L.orc_eos_e(p, x[0], x[1]) + P / x[0]) / h_in - 1.0]

    rho_in, T_in = optimize.fsolve(res, [2.0 / (3.0 * b), 1.5 * Tc], xtol=1e-13)
    return wl.Case(name="throttle", dim=3, nx=1, ny=1, nz=40, zwalls=2, eos="vdw", R=1.0, cv=cv, a=a, b=b,
                   k_over_mu=0.35, eta_over_mu=3.0, tau_f=2.0, tau_g=2.0, phi_central=1, face_kind=(5, 3),
                   face_P=(P_in, 0.98 * P_in), Tw_lo=T_in, Tw_hi=T_in, throttle_K=0.02, throttle_sigma=3.0,
                   storage=storage, init=dict(kind="duct", rho0=rho_in, u0=0.0, T0=T_in))


@pytest.mark.parametrize("variant", [SPLIT, (ZMARCH, (30, 6, 4))])
@pytest.mark.parametrize("storage,tol,steps", [("f64", 1e-12, 300), ("f32", 1e-5, 60)])
def test_throttle_matches_oracle(storage, tol, steps, variant):
    # float32 over fewer steps: in this dense, cold fluid (theta ~ 0.016, b rho ~ 0.66) the pressure and
    # the boundary Newton steps lose digits to cancellation, and the weakly damped sound waves carry the
    # rounding along: float32 drifts to 2e-5 of the float64 oracle by 300 steps
    c = _throttle_case(storage)
    sim, o = _pair(c, steps, _noisy_fields(c, 0.002, 34), variant)
    _compare(sim, o, tol, f32=storage == "f32")


def test_throttle_joule_thomson_on_the_gpu():
    # steady throttling: Delta T / Delta P equals the van der Waals Joule-Thomson coefficient
    c = _throttle_case("f64")
    sim = lbm.Simulation(c)
    sim.init()
    sim.step(25000)
    rho, u, T = sim.moments()
    o = orc.Oracle(oracle_params(c))
    L = orc.lib()
    P = np.array([L.orc_eos_P(o.p, r, t) for r, t in zip(rho, T)])
    r_m, T_m = 0.5 * (rho[1] + rho[-2]), 0.5 * (T[1] + T[-2])
    P_rho, P_T = L.orc_eos_dPdrho(o.p, r_m, T_m), L.orc_eos_dPdT(o.p, r_m, T_m)
    c_P = L.orc_eos_cv(o.p, r_m, T_m) + T_m * P_T ** 2 / (r_m ** 2 * P_rho)
    mu_jt = -(1.0 / r_m - T_m * P_T / (r_m ** 2 * P_rho)) / c_P
    assert (T[-2] - T[1]) / (P[-2] - P[1]) == pytest.approx(mu_jt, rel=0.02)


# Supersonic inlet (Ma 1.5; static inlet, extrapolated outlet, the upwind-biased Phi), the
# window in which uniform supersonic flow of this step is stable: T_in 0.02, tau 1.
SS_T, SS_U = 0.02, 1.5 * math.sqrt(GAM * R_GAS * 0.02)


def _ss_duct(nz=50, nx=1, ny=1, q=0.0, friction=0.0, storage="f64"):
    return wl.Case(name="ss_duct", dim=3, nx=nx, ny=ny, nz=nz, zwalls=2, eos="ideal", R=R_GAS, cv=CV,
                   k_over_mu=CP / 0.71, tau_f=1.0, tau_g=1.0, phi_central=0, q=q, zlo=0, zhi=0, friction=friction,
                   face_kind=(2, 4), face_P=(SS_T, 0.0), uw_lo=(0.0, 0.0, SS_U), Tw_lo=SS_T, Tw_hi=SS_T,
                   storage=storage, init=dict(kind="duct", rho0=1.0, u0=SS_U, T0=SS_T))


@pytest.mark.parametrize("q,friction", [(8e-7, 0.0), (0.0, 5e-4)], ids=["rayleigh", "fanno"])
@pytest.mark.parametrize("variant", [SPLIT, (ZMARCH, (30, 6, 32))])
def test_supersonic_duct_parity(q, friction, variant):
    c = _ss_duct(q=q, friction=friction)
    fields = _noisy_fields(c, 1e-3, 41)
    sim, o = _pair(c, 300, fields, variant)
    _compare(sim, o, 1e-12)


@pytest.mark.parametrize("q,friction", [(8e-7, 0.0), (0.0, 5e-4)], ids=["rayleigh", "fanno"])
def test_supersonic_duct_parity_bundle(q, friction):
    # a 4 x 3 bundle of ducts (transverse velocities from the noise) in float64 on the z-march
    # with extrapolated faces
    c = _ss_duct(nx=4, ny=3, q=q, friction=friction)
    fields = _noisy_fields(c, 1e-3, 42)
    sim, o = _pair(c, 300, fields, (ZMARCH, (30, 6, 32)))
    _compare(sim, o, 1e-12)


@pytest.mark.parametrize("q,friction", [(8e-7, 0.0), (0.0, 5e-4)], ids=["rayleigh", "fanno"])
@pytest.mark.parametrize("variant", [SPLIT, (ZMARCH, (30, 6, 32))])
def test_supersonic_duct_parity_f32(q, friction, variant):
    # float32 on a single column: u_z > 0 everywhere and no transverse velocity, so the
    # upwind-biased branch is the same as in float64 (in a bundle, noise-driven transverse
    # velocities round across zero and take the other branch in some cells)
    # At Ma 1.5 the uniform state has a weakly growing mode (spectral radius lam of the
    # one-step amplification, from the oracle's own linearisation): float32 rounding
    # (<= 2^-24 per step) grows by at most sum_k lam^k over n steps.
    from oracle import stability as st

    n = 300
    c = _ss_duct(q=q, friction=friction, storage="f32")
    _, r, _ = st.amplification(st.column_case(c, 16), 1.0, (0.0, 0.0, SS_U), SS_T)
    lam = float(np.max(r))
    tol = 1e-5 + 2.0 ** -24 * (lam ** n - 1.0) / (lam - 1.0)
    fields = _noisy_fields(c, 1e-3, 42)
    sim, o = _pair(c, n, fields, variant)
    _compare(sim, o, tol, f32=True)
