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
