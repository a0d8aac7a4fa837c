"""Helpers shared by the tests: oracle parameters from a workload case."""
import numpy as np

from oracle import oracle as orc


def oracle_params(case):
    return orc.params_from_case(case)


def run_oracle(case, steps, fields=None):
    o = orc.Oracle(oracle_params(case))
    rho, u, T = fields if fields is not None else case.fields()
    o.init(rho, u, T)
    o.step(steps)
    return o


def rel_linf(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))


def maxwell(eos, T, guess=(1.5, 5.8)):
    """Coexistence densities (rho_v, rho_l) at T by the equal-area construction on
    the oracle's own pressure: P(rho_v) = P(rho_l) = P_s and
    int_{1/rho_l}^{1/rho_v} P dv = P_s (1/rho_v - 1/rho_l)."""
    from scipy import integrate, optimize

    def resid(x):
        rv, rl = x
        Ps = eos.P(rl, T)
        area = integrate.quad(lambda r: eos.P(r, T) / (r * r), rv, rl, epsabs=1e-13)[0]
        return [eos.P(rv, T) - Ps, area - Ps * (1 / rv - 1 / rl)]

    return optimize.fsolve(resid, list(guess), xtol=1e-12)
