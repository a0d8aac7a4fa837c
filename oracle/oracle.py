"""ctypes wrapper of the FP64 CPU oracle (``lbm_oracle.c``).

Test infrastructure only: the test suite, the smoke check and the CPU-baseline
leg of the benchmark use it to produce the values the CUDA path must match.
The product library never imports it.

Field layout matches the library's host-side convention: scalars are ``[N]``
and vectors ``[dim][N]`` float64 arrays, cell index ``x + nx*(y + ny*z)``.
Populations are ``[Q][N]``; direction ``i`` has base-3 digits
``(d_x, d_y, d_z)`` with digit 0, 1, 2 meaning c = 0, +1, -1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

IDEAL, VDW, PR = 0, 1, 2
_EOS_NAMES = {"ideal": IDEAL, "vdw": VDW, "pr": PR}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-std=c11", "-Wall", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("zwalls", ctypes.c_int), ("eos", ctypes.c_int),
        ("R", ctypes.c_double), ("cv", ctypes.c_double),
        ("a", ctypes.c_double), ("b", ctypes.c_double),
        ("Tc", ctypes.c_double), ("omega", ctypes.c_double),
        ("kappa", ctypes.c_double), ("eta_over_mu", ctypes.c_double), ("k_over_mu", ctypes.c_double),
        ("tau_f", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("accel", ctypes.c_double * 3),
        ("q", ctypes.c_double), ("zlo", ctypes.c_int), ("zhi", ctypes.c_int),
        ("phi_central", ctypes.c_int),
        ("mu", ctypes.c_double),
        ("isothermal", ctypes.c_int),
        ("uw_lo", ctypes.c_double * 3), ("uw_hi", ctypes.c_double * 3),
        ("Tw_lo", ctypes.c_double), ("Tw_hi", ctypes.c_double),
        ("wall_rho", ctypes.c_int),
        ("face_kind", ctypes.c_int * 2), ("face_P", ctypes.c_double * 2),
        ("friction", ctypes.c_double),
        ("throttle_K", ctypes.c_double), ("throttle_sigma", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, vp, dp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(OrcParams)
        sig = {
            "orc_lattice": (i, [i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
            "orc_psi": (d, [i, d, d]),
            "orc_fprod": (None, [i, d, dp, dp, dp]),
            "orc_geq": (None, [i, d, dp, d, d, dp]),
            "orc_eos_P": (d, [pp, d, d]),
            "orc_eos_e": (d, [pp, d, d]),
            "orc_eos_dPdT": (d, [pp, d, d]),
            "orc_eos_dPdrho": (d, [pp, d, d]),
            "orc_eos_cv": (d, [pp, d, d]),
            "orc_eos_T": (d, [pp, d, d, d, ctypes.POINTER(ctypes.c_int)]),
            "orc_vdw_from_critical": (None, [d, d, d, dp, dp]),
            "orc_pr_from_critical": (None, [d, d, d, dp, dp]),
            "orc_create": (vp, [pp]),
            "orc_destroy": (None, [vp]),
            "orc_set_threads": (None, [i]),
            "orc_get_threads": (i, []),
            "orc_init": (i, [vp, dp, dp, dp]),
            "orc_step": (i, [vp, i]),
            "orc_set_accel": (None, [vp, dp]),
            "orc_set_fields": (None, [vp, dp, dp]),
            "orc_moments": (i, [vp, dp, dp, dp]),
            "orc_invariants": (i, [vp, dp]),
            "orc_populations": (i, [vp, dp, dp]),
            "orc_set_populations": (i, [vp, dp, dp, dp]),
            "orc_newton_cap_hits": (ctypes.c_long, [vp]),
            "orc_theta_nonpositive": (ctypes.c_long, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(dim=2, nx=8, ny=8, nz=1, zwalls=0, eos="ideal", R=1.0, cv=2.5, a=0.0, b=0.0,
                Tc=1.0, omega=0.0, Pc=None, kappa=0.0, eta_over_mu=0.0, k_over_mu=0.0,
                tau_f=0.8, tau_g=0.8, accel=(0.0, 0.0, 0.0), q=0.0, zlo=0, zhi=0,
                phi_central=0, mu=0.0, isothermal=0, uw_lo=(0.0, 0.0, 0.0), uw_hi=(0.0, 0.0, 0.0),
                Tw_lo=0.0, Tw_hi=0.0, wall_rho=0, face_kind=(0, 0), face_P=(0.0, 0.0), friction=0.0, throttle_K=0.0,
                throttle_sigma=0.0) -> OrcParams:
    """Build the oracle's parameter struct.  For Peng-Robinson with ``Pc`` given
    and ``a == 0``, a and b follow from (Tc, Pc) by the oracle's own helper.
    zwalls = 2 selects the non-equilibrium-extrapolation walls with wall
    velocities uw_lo, uw_hi and temperatures Tw_lo, Tw_hi; wall_rho picks the
    boundary density (0: from the neighbour's pressure, 1: the neighbour's)."""
    kind = _EOS_NAMES[eos] if isinstance(eos, str) else int(eos)
    if kind == PR and a == 0.0 and Pc is not None:
        a, b = pr_from_critical(R, Tc, Pc)
    p = OrcParams()
    p.dim, p.nx, p.ny, p.nz, p.zwalls, p.eos = dim, nx, ny, nz, zwalls, kind
    p.R, p.cv, p.a, p.b, p.Tc, p.omega = R, cv, a, b, Tc, omega
    p.kappa, p.eta_over_mu, p.k_over_mu = kappa, eta_over_mu, k_over_mu
    p.tau_f, p.tau_g = tau_f, tau_g
    for k in range(3):
        p.accel[k] = accel[k] if k < len(accel) else 0.0
    p.q, p.zlo, p.zhi = q, zlo, zhi
    p.phi_central = int(phi_central)
    p.mu = float(mu)
    p.isothermal = int(isothermal)
    for k in range(3):
        p.uw_lo[k] = uw_lo[k] if k < len(uw_lo) else 0.0
        p.uw_hi[k] = uw_hi[k] if k < len(uw_hi) else 0.0
    p.Tw_lo, p.Tw_hi = float(Tw_lo), float(Tw_hi)
    p.wall_rho = int(wall_rho)
    for f in range(2):
        p.face_kind[f] = int(face_kind[f])
        p.face_P[f] = float(face_P[f])
    p.friction = float(friction)
    p.throttle_K, p.throttle_sigma = float(throttle_K), float(throttle_sigma)
    return p


def lattice(dim: int):
    c = (ctypes.c_int * 81)()
    opp = (ctypes.c_int * 27)()
    Q = lib().orc_lattice(dim, c, opp)
    cv = np.array(c[: 3 * Q], dtype=np.int64).reshape(Q, 3)[:, :dim]
    return cv, np.array(opp[:Q], dtype=np.int64)


def psi(c: int, xi: float, zeta: float) -> float:
    return lib().orc_psi(c, xi, zeta)


def fprod(dim: int, rho: float, xi, zeta) -> np.ndarray:
    Q = 3 ** dim
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    zeta = np.ascontiguousarray(zeta, dtype=np.float64)
    out = np.zeros(Q)
    lib().orc_fprod(dim, rho, _dp(xi), _dp(zeta), _dp(out))
    return out


def feq(dim: int, rho: float, u, theta: float) -> np.ndarray:
    u = np.asarray(u, dtype=np.float64)
    return fprod(dim, rho, u, theta + u * u)


def geq(dim: int, rho: float, u, e: float, theta: float) -> np.ndarray:
    Q = 3 ** dim
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    lib().orc_geq(dim, rho, _dp(u), e, theta, _dp(out))
    return out


class EoS:
    """Equation-of-state functions of the oracle for one parameter set."""

    def __init__(self, params: OrcParams):
        self.p = params

    def P(self, rho, T):
        return lib().orc_eos_P(ctypes.byref(self.p), rho, T)

    def e(self, rho, T):
        return lib().orc_eos_e(ctypes.byref(self.p), rho, T)

    def dPdT(self, rho, T):
        return lib().orc_eos_dPdT(ctypes.byref(self.p), rho, T)

    def dPdrho(self, rho, T):
        return lib().orc_eos_dPdrho(ctypes.byref(self.p), rho, T)

    def cv(self, rho, T):
        return lib().orc_eos_cv(ctypes.byref(self.p), rho, T)

    def T(self, rho, e, T_guess=0.0):
        it = ctypes.c_int(0)
        T = lib().orc_eos_T(ctypes.byref(self.p), rho, e, T_guess, ctypes.byref(it))
        return T, it.value


def vdw_from_critical(R, Tc, Pc):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_vdw_from_critical(R, Tc, Pc, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def pr_from_critical(R, Tc, Pc):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_pr_from_critical(R, Tc, Pc, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


class Oracle:
    """One simulation on the CPU oracle."""

    def __init__(self, params: OrcParams):
        self.p = params
        self.dim = params.dim
        self.N = params.nx * params.ny * params.nz
        self.Q = 3 ** params.dim
        self._h = lib().orc_create(ctypes.byref(params))
        if not self._h:
            raise ValueError("oracle: invalid parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init(self, rho, u, T):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.N)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.dim, self.N)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.N)
        lib().orc_init(self._h, _dp(rho), _dp(u), _dp(T))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros((self.dim, self.N))
        T = np.zeros(self.N)
        lib().orc_moments(self._h, _dp(rho), _dp(u), _dp(T))
        return rho, u, T

    def invariants(self) -> np.ndarray:
        out = np.zeros(2 * self.dim + 3)
        lib().orc_invariants(self._h, _dp(out))
        return out

    def set_fields(self, F=None, Q=None):
        """Per-cell body force F_B [dim][N] and heat source Q [N] (None: none)."""
        Fp = Qp = None
        if F is not None:
            F = np.ascontiguousarray(F, dtype=np.float64).reshape(self.dim, self.N)
            Fp = _dp(F)
        if Q is not None:
            Q = np.ascontiguousarray(Q, dtype=np.float64).reshape(self.N)
            Qp = _dp(Q)
        lib().orc_set_fields(self._h, Fp, Qp)

    def set_accel(self, accel):
        a = np.ascontiguousarray(np.asarray(accel, dtype=np.float64).reshape(-1)[:3])
        if a.size < 3:
            a = np.concatenate([a, np.zeros(3 - a.size)])
        lib().orc_set_accel(self._h, _dp(a))

    def populations(self):
        f = np.zeros((self.Q, self.N))
        g = np.zeros((self.Q, self.N))
        lib().orc_populations(self._h, _dp(f), _dp(g))
        return f, g

    def set_populations(self, f, g, T_guess=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        tg = None if T_guess is None else _dp(np.ascontiguousarray(T_guess, dtype=np.float64))
        lib().orc_set_populations(self._h, _dp(f), _dp(g), tg)

    @property
    def newton_cap_hits(self) -> int:
        return int(lib().orc_newton_cap_hits(self._h))

    @property
    def theta_nonpositive(self) -> int:
        return int(lib().orc_theta_nonpositive(self._h))


def params_from_case(case) -> OrcParams:
    """Oracle parameters of a workload case (paper_2609_28679_b300.workloads.Case)."""
    a, b = case.a, case.b
    if case.eos == "pr" and a == 0.0:
        a, b = pr_from_critical(case.R, case.Tc, case.Pc)
    return make_params(dim=case.dim, nx=case.nx, ny=case.ny, nz=case.nz, zwalls=case.zwalls,
                       eos=case.eos, R=case.R, cv=case.cv, a=a, b=b, Tc=case.Tc, omega=case.omega,
                       kappa=case.kappa, eta_over_mu=case.eta_over_mu, k_over_mu=case.k_over_mu,
                       tau_f=case.tau_f, tau_g=case.tau_g, accel=case.accel, q=case.q,
                       zlo=case.zlo, zhi=case.zhi, phi_central=case.phi_central, mu=getattr(case, "mu", 0.0),
                       isothermal=getattr(case, "isothermal", 0), uw_lo=getattr(case, "uw_lo", (0.0, 0.0, 0.0)),
                       uw_hi=getattr(case, "uw_hi", (0.0, 0.0, 0.0)), Tw_lo=getattr(case, "Tw_lo", 0.0),
                       Tw_hi=getattr(case, "Tw_hi", 0.0), wall_rho=getattr(case, "wall_rho", 0),
                       face_kind=getattr(case, "face_kind", (0, 0)), face_P=getattr(case, "face_P", (0.0, 0.0)),
                       friction=getattr(case, "friction", 0.0), throttle_K=getattr(case, "throttle_K", 0.0),
                       throttle_sigma=getattr(case, "throttle_sigma", 0.0))
