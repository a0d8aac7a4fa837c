"""Pins of the oracle's equations of state (Eqs. idealEOS, vdw_eos, de_rho,
TdependsongenericEOS, JT_coeff; Peng-Robinson in its textbook form) against
critical-point conditions, the paper's nitrogen table, finite differences,
quadrature of the caloric relation and closed-form inversions."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _eos(kind):
    if kind == "ideal":
        return orc.EoS(orc.make_params(eos="ideal", R=1.0, cv=2.5))
    if kind == "vdw":
        return orc.EoS(orc.make_params(eos="vdw", R=1.0, cv=2.5, a=9 / 49, b=2 / 21))
    a, b = orc.pr_from_critical(1.0, 0.5, 0.1537005)
    return orc.EoS(orc.make_params(eos="pr", R=1.0, cv=2.5, a=a, b=b, Tc=0.5, omega=0.1))


STATES = {"ideal": [(0.5, 0.3), (1.3, 0.7)],
          "vdw": [(1.0, 0.5), (3.5, 0.55), (5.5, 0.52)],
          "pr": [(0.3, 0.475), (1.0, 0.45), (2.1, 0.46)]}


def test_vdw_critical_point_exact():
    # a = 27 R^2 Tc^2/(64 Pc), b = R Tc/(8 Pc): the critical isotherm has a horizontal
    # inflection at rho_c = 1/(3b) with P = Pc (Z_c = 3/8).
    R, Tc, Pc = 1.0, 4.0 / 7.0, 0.75
    a, b = orc.vdw_from_critical(R, Tc, Pc)
    assert a == pytest.approx(9 / 49, rel=1e-14) and b == pytest.approx(2 / 21, rel=1e-14)
    eos = orc.EoS(orc.make_params(eos="vdw", R=R, cv=2.5, a=a, b=b))
    rc = 1.0 / (3.0 * b)
    assert eos.P(rc, Tc) == pytest.approx(Pc, rel=1e-13)
    assert abs(eos.dPdrho(rc, Tc)) < 1e-13
    h = 1e-4
    d2 = (eos.dPdrho(rc + h, Tc) - eos.dPdrho(rc - h, Tc)) / (2 * h)
    assert abs(d2) < 1e-7


def test_nitrogen_table_critical_density():
    vals = {}
    with open(os.path.join(GOLDEN, "nitrogen_critical.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    R = 8.314462618 / 0.0280134
    a, b = orc.vdw_from_critical(R, vals["Tc_K"], vals["Pc_Pa"])
    eos = orc.EoS(orc.make_params(eos="vdw", R=R, cv=R / vals["R_over_cv"], a=a, b=b))
    rc = 1.0 / (3.0 * b)
    assert rc == pytest.approx(vals["rho_c_kg_m3"], rel=1e-3)
    assert abs(eos.dPdrho(rc, vals["Tc_K"])) < 1e-9 * R * vals["Tc_K"]


def test_pr_critical_point_textbook():
    # Peng-Robinson's Omega_a = 0.45724, Omega_b = 0.07780 encode the critical conditions
    # with Z_c = 0.3074 (to the 5 digits of the constants).
    R, Tc, Pc = 1.0, 0.5, 0.1537005
    eos = _eos("pr")
    rho = np.linspace(0.6, 1.4, 80001)
    slope = np.array([eos.dPdrho(r, Tc) for r in rho])
    k = int(np.argmin(slope))
    rho_star = rho[k]
    assert abs(slope[k]) < 1e-3 * R * Tc
    assert rho_star == pytest.approx(Pc / (0.3074 * R * Tc), rel=2e-3)
    assert eos.P(rho_star, Tc) == pytest.approx(Pc, rel=1e-3)


@pytest.mark.parametrize("kind", ["ideal", "vdw", "pr"])
def test_derivatives_match_finite_differences(kind):
    eos = _eos(kind)
    for rho, T in STATES[kind]:
        hT, hr = 1e-6 * T, 1e-6 * rho
        dPdT = (eos.P(rho, T + hT) - eos.P(rho, T - hT)) / (2 * hT)
        dPdr = (eos.P(rho + hr, T) - eos.P(rho - hr, T)) / (2 * hr)
        cv = (eos.e(rho, T + hT) - eos.e(rho, T - hT)) / (2 * hT)
        assert eos.dPdT(rho, T) == pytest.approx(dPdT, rel=1e-8, abs=1e-10)
        assert eos.dPdrho(rho, T) == pytest.approx(dPdr, rel=1e-8, abs=1e-10)
        assert eos.cv(rho, T) == pytest.approx(cv, rel=1e-8)


@pytest.mark.parametrize("kind", ["ideal", "vdw", "pr"])
def test_caloric_relation_by_quadrature(kind):
    # Eq. de_rho at constant T: e(rho,T) - e(0,T) = -int_0^rho [T dP/dT - P] / r^2 dr, e(0,T) = cv T.
    eos = _eos(kind)
    for rho, T in STATES[kind]:
        integrand = lambda r: (T * eos.dPdT(r, T) - eos.P(r, T)) / (r * r)
        val, err = integrate.quad(integrand, 1e-12, rho, epsabs=1e-13, epsrel=1e-12)
        assert eos.e(rho, T) - 2.5 * T == pytest.approx(-val, rel=1e-9, abs=1e-11)


@pytest.mark.parametrize("kind", ["ideal", "vdw", "pr"])
def test_temperature_inversion_round_trip(kind):
    eos = _eos(kind)
    for rho, T in STATES[kind]:
        e = eos.e(rho, T)
        Tn, it = eos.T(rho, e, T_guess=T * 1.05)
        assert Tn == pytest.approx(T, rel=1e-13)
        assert it < 50


def test_pr_newton_matches_closed_form():
    # With constant cv and the Soave alpha, e is quadratic in s = sqrt(T/Tc):
    #   cv Tc s^2 + a k (1+k) L s - [a (1+k)^2 L + e] = 0,  L = int_0^rho dr/(1 + 2br - b^2 r^2),
    # so the positive root gives T exactly; Newton must land on it.
    a, b = orc.pr_from_critical(1.0, 0.5, 0.1537005)
    eos = _eos("pr")
    k = 0.37464 + 1.54226 * 0.1 - 0.26992 * 0.01
    for rho, e in [(0.3, 0.6), (1.0, 0.2), (2.1, -0.4), (0.26, 1.0)]:
        L = integrate.quad(lambda r: 1.0 / (1 + 2 * b * r - b * b * r * r), 0.0, rho, epsabs=1e-14, epsrel=1e-13)[0]
        A, B, C = 2.5 * 0.5, a * k * (1 + k) * L, a * (1 + k) ** 2 * L + e
        s = (-B + math.sqrt(B * B + 4 * A * C)) / (2 * A)
        T_exact = 0.5 * s * s
        Tn, it = eos.T(rho, e, T_guess=0.45)
        assert Tn == pytest.approx(T_exact, rel=1e-12)


def test_joule_thomson_inversion_vdw():
    # Eq. JT_coeff: mu_JT = -(1/C_P)[1/rho - T dP/dT /(rho^2 dP/drho)] vanishes for an ideal gas and,
    # for van der Waals, changes sign on the inversion curve T_inv = 2a (1 - b rho)^2 / (R b).
    def mu_jt_times_cp(eos, rho, T):
        return -(1.0 / rho - T * eos.dPdT(rho, T) / (rho * rho * eos.dPdrho(rho, T)))

    ideal = _eos("ideal")
    for rho, T in [(0.5, 0.3), (2.0, 1.0)]:
        assert abs(mu_jt_times_cp(ideal, rho, T)) < 1e-15
    vdw = _eos("vdw")
    a, b = 9 / 49, 2 / 21
    for rho in [0.2, 0.8, 1.5]:
        Tinv = 2 * a * (1 - b * rho) ** 2 / b
        lo = mu_jt_times_cp(vdw, rho, Tinv * (1 - 1e-3))
        hi = mu_jt_times_cp(vdw, rho, Tinv * (1 + 1e-3))
        assert lo > 0 > hi
