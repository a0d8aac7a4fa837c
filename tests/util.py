"""Helpers shared by the tests: oracle parameters from a workload case."""
import numpy as np

from oracle import oracle as orc


def oracle_params(case):
    a, b = case.a, case.b
    if case.eos == "pr" and a == 0.0:
        a, b = orc.pr_from_critical(case.R, case.Tc, case.Pc)
    return orc.make_params(dim=case.dim, nx=case.nx, ny=case.ny, nz=case.nz, zwalls=case.zwalls,
                           eos=case.eos, R=case.R, cv=case.cv, a=a, b=b, Tc=case.Tc, omega=case.omega,
                           kappa=case.kappa, eta_over_mu=case.eta_over_mu, k_over_mu=case.k_over_mu,
                           tau_f=case.tau_f, tau_g=case.tau_g, accel=case.accel, q=case.q,
                           zlo=case.zlo, zhi=case.zhi, phi_central=case.phi_central)


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
