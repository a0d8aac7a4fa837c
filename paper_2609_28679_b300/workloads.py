"""Seeded synthetic inputs shaped like the paper's test cases.

This module holds the workload recipes only (grid sizes, parameters, initial
fields, seeded noise); it contains none of the method's arithmetic.  Both the
CUDA path and the CPU oracle receive the same host arrays from here.

Random numbers come from a counter-based generator: splitmix64 of
``seed XOR linear_index`` mapped to a uniform double in [-1, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [-1, 1): splitmix64(seed ^ index), top 53 bits."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    z = splitmix64(idx ^ np.uint64(seed))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 / 2.0 ** 53) - 1.0


@dataclass
class Case:
    """One simulation: lattice, fluid, relaxation, sources and initial fields."""
    name: str
    dim: int
    nx: int
    ny: int
    nz: int = 1
    zwalls: int = 0
    eos: str = "ideal"            # ideal | vdw | pr
    R: float = 1.0
    cv: float = 2.5
    a: float = 0.0
    b: float = 0.0
    Tc: float = 1.0
    Pc: float = 0.0
    omega: float = 0.0
    kappa: float = 0.0
    eta_over_mu: float = 0.0
    k_over_mu: float = 0.0
    tau_f: float = 0.8
    tau_g: float = 0.8
    accel: tuple = (0.0, 0.0, 0.0)
    q: float = 0.0
    zlo: int = 0
    zhi: int = 0                  # <= 0: heat source everywhere
    phi_central: int = 0          # derivative in the Galilean correction: 0 upwind-biased, 1 central
    mu: float = 0.0               # > 0: tau = mu / P per cell (one tau for f and g); 0: tau_f, tau_g
    isothermal: int = 0           # 1: g not evolved, every cell keeps its initial T
    t_solver: int = 0             # Peng-Robinson T(rho, e): 0 Newton, 1 learned start + Newton
    uw_lo: tuple = (0.0, 0.0, 0.0)  # zwalls = 2 (non-equilibrium-extrapolation walls on z = 0, nz - 1):
    uw_hi: tuple = (0.0, 0.0, 0.0)  # wall velocities,
    Tw_lo: float = 0.0              # wall temperatures,
    Tw_hi: float = 0.0
    wall_rho: int = 0               # and boundary density: 0 from the neighbour's pressure, 1 the neighbour's,
                                    # 2 from the pressure extrapolated linearly from two cells inside
    face_kind: tuple = (0, 0)       # zwalls = 2, per face: 0 wall, 1 inlet (total P0 = face_P, T0 = Tw),
                                    # 2 inlet (static P = face_P, T = Tw, u = uw), 3 outlet (static P), 4 outlet
                                    # (extrapolated), 5 inlet (static P = face_P, T = Tw, u of the neighbour)
    face_P: tuple = (0.0, 0.0)      # pressure datum of each open face
    friction: float = 0.0           # duct friction k = f_D / (2 D_h): F = -k rho |u| u, Q = -F.u
    throttle_K: float = 0.0         # throttle: F = -K phi(z) rho u, Q = -F.u, phi a Gaussian of width
    throttle_sigma: float = 0.0     # throttle_sigma at the middle of the duct (dim 3)
    storage: str = "f64"          # f64 | f32 | bf16 | f16
    steps: int = 100
    init: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def fields(self):
        """Initial (rho [N], u [dim][N], T [N]) as float64 arrays."""
        return _FIELDS[self.init["kind"]](self)


def _coords(c: Case):
    z, y, x = np.meshgrid(np.arange(c.nz), np.arange(c.ny), np.arange(c.nx), indexing="ij")
    return x.ravel().astype(np.float64), y.ravel().astype(np.float64), z.ravel().astype(np.float64)


def _waves(c: Case):
    """rho = rho0 (1 + A_rho sin(2 pi x / nx)), u_y = A_u sin(2 pi x / nx), uniform T."""
    x, _, _ = _coords(c)
    s = np.sin(2.0 * math.pi * x / c.nx)
    rho = c.init.get("rho0", 1.0) * (1.0 + c.init.get("amp_rho", 0.0) * s)
    u = np.zeros((c.dim, c.ncell))
    u[1] = c.init.get("amp_u", 0.0) * s
    T = np.full(c.ncell, c.init.get("T0", 0.3))
    return rho, u, T


def _noisy_density(c: Case):
    """rho = rho0 (1 + amp * xi), xi ~ U[-1,1) seeded; u = 0; uniform T."""
    xi = uniform_pm1(c.init["seed"], c.ncell)
    rho = c.init["rho0"] * (1.0 + c.init["amp"] * xi)
    return rho, np.zeros((c.dim, c.ncell)), np.full(c.ncell, c.init["T0"])


def _noisy_temperature(c: Case):
    """uniform rho0; T = T0 (1 + amp * xi) seeded; u = 0."""
    xi = uniform_pm1(c.init["seed"], c.ncell)
    T = c.init["T0"] * (1.0 + c.init["amp"] * xi)
    return np.full(c.ncell, c.init["rho0"]), np.zeros((c.dim, c.ncell)), T


def _droplet(c: Case):
    """Centred droplet, tanh profile of half-width w, noise on the interface shell."""
    x, y, z = _coords(c)
    cx, cy, cz = (c.nx - 1) / 2.0, (c.ny - 1) / 2.0, (c.nz - 1) / 2.0
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + ((z - cz) ** 2 if c.dim == 3 else 0.0))
    R0, w = c.init["radius"], c.init.get("width", 2.0)
    rl, rv = c.init["rho_l"], c.init["rho_v"]
    rho = rv + (rl - rv) * 0.5 * (1.0 - np.tanh((r - R0) / w))
    xi = uniform_pm1(c.init["seed"], c.ncell)
    shell = np.abs(r - R0) < c.init.get("shell", 4.0)
    rho = np.where(shell, rho * (1.0 + c.init.get("amp", 0.01) * xi), rho)
    return rho, np.zeros((c.dim, c.ncell)), np.full(c.ncell, c.init["T0"])


def _couette(c: Case):
    """Linear u_x and T between the wall cells z = 0 and z = nz - 1 (their
    wall values), rho = rho_ref T_ref / T (uniform rho T), plus seeded noise of
    relative size amp on rho (default 0)."""
    _, _, z = _coords(c)
    s = z / (c.nz - 1)
    T = c.Tw_lo + (c.Tw_hi - c.Tw_lo) * s
    u = np.zeros((c.dim, c.ncell))
    for a in range(c.dim):
        u[a] = c.uw_lo[a] + (c.uw_hi[a] - c.uw_lo[a]) * s
    rho = c.init.get("rho0", 1.0) * c.Tw_lo / T
    amp = c.init.get("amp", 0.0)
    if amp:
        rho = rho * (1.0 + amp * uniform_pm1(c.init.get("seed", 1), c.ncell))
    return rho, u, T


def _duct(c: Case):
    """Uniform rho0, T0 and velocity u0 along the last axis (the duct axis)."""
    u = np.zeros((c.dim, c.ncell))
    u[c.dim - 1] = c.init.get("u0", 0.0)
    return (np.full(c.ncell, c.init.get("rho0", 1.0)), u, np.full(c.ncell, c.init.get("T0", 0.3)))


def _uniform(c: Case):
    return (np.full(c.ncell, c.init.get("rho0", 1.0)), np.zeros((c.dim, c.ncell)),
            np.full(c.ncell, c.init.get("T0", 0.3)))


_FIELDS = {"waves": _waves, "noisy_density": _noisy_density, "noisy_temperature": _noisy_temperature,
           "droplet": _droplet, "uniform": _uniform, "couette": _couette, "duct": _duct}

# van der Waals fluid of the 2-D multiphase cases.  b = 2/21 (rho_c = 3.5) and
# R/c_v = 0.4 as in the nitrogen table; a = 9/245 puts Tc = 4/35, i.e. the
# fluid with a = 9/49 run with a time step sqrt(5) smaller, so that the
# Maxwell liquid's adiabatic sound speed (0.54) stays below the lattice speed
# (with a = 9/49 it is 1.21 and every run diverges).  Capillarity and gravity
# scale with a: kappa = 0.1/5, g = 1e-6/5.
VDW_SCALE = 0.2
VDW_A, VDW_B, VDW_RHOC = 9.0 / 49.0 * VDW_SCALE, 2.0 / 21.0, 3.5
VDW_TC = 8.0 * VDW_A / (27.0 * VDW_B)
VDW_KAPPA, VDW_G, VDW_ETA = 0.1 * VDW_SCALE, 1e-6 * VDW_SCALE, 3.0
# Mean of the Maxwell densities at T/Tc = 0.9 (vapour 1.490096, liquid 5.800446).
VDW_RHO_MID_090 = 3.6452707
# Peng-Robinson fluid of the heated slab: Tc = 0.5, Pc chosen so that rho_c ~ 1, omega = 0.1.
PR_TC, PR_PC, PR_OMEGA = 0.5, 0.1537005, 0.1
# The droplet holds Maxwell liquid (rho_l = 2.10988 at T/Tc = 0.9), whose
# adiabatic sound speed at Tc = 0.5 is 1.33 lattice speeds; it runs with the
# temperature scale 20x smaller (time step sqrt(20) smaller): Tc = 0.025,
# kappa, Q scaled likewise, and bulk viscosity eta/mu = 10 to damp the
# acoustic modes of the liquid.
PR_DROP_SCALE = 0.05


def acoustic_shear(n: int = 128, steps: int = 1000, storage: str = "f64") -> Case:
    """2-D periodic ideal gas (gamma = 1.4): density pulse plus shear wave,
    constant body force and uniform heat source."""
    return Case(name=f"acoustic_shear_{n}", dim=2, nx=n, ny=n, eos="ideal", R=1.0, cv=2.5,
                k_over_mu=3.5 / 0.71, accel=(1e-5, 0.0, 0.0), q=1e-6, storage=storage, steps=steps,
                init=dict(kind="waves", rho0=1.0, amp_rho=1e-3, amp_u=1e-3, T0=0.3))


def vdw_spinodal(n: int = 512, steps: int = 20000, storage: str = "f32", Tr: float = 0.9,
                 rho0: float = VDW_RHO_MID_090, seed: int = 2, ny: int | None = None) -> Case:
    """2-D periodic van der Waals quench at T/Tc = Tr with Korteweg capillarity
    and gravity; rho0 defaults to the mean of the Maxwell densities at Tr = 0.9."""
    return Case(name=f"vdw_spinodal_{n}", dim=2, nx=n, ny=ny or n, eos="vdw", R=1.0, cv=2.5,
                a=VDW_A, b=VDW_B, kappa=VDW_KAPPA, eta_over_mu=VDW_ETA, k_over_mu=3.5,
                accel=(0.0, -VDW_G, 0.0), phi_central=1, storage=storage, steps=steps,
                init=dict(kind="noisy_density", rho0=rho0, amp=0.01, T0=Tr * VDW_TC, seed=seed))


def pr_heated_slab(n: int = 256, steps: int = 5000, storage: str = "f32", nz: int | None = None) -> Case:
    """3-D Peng-Robinson slab at T/Tc = 0.95, periodic in x and y, bounce-back
    walls in z, gravity, heat source in the bottom 10 % of z."""
    nz = nz or n
    return Case(name=f"pr_heated_slab_{n}", dim=3, nx=n, ny=n, nz=nz, zwalls=1, eos="pr", R=1.0,
                cv=2.5, Tc=PR_TC, Pc=PR_PC, omega=PR_OMEGA, kappa=0.2, k_over_mu=3.5,
                accel=(0.0, 0.0, -1e-5), q=1e-6, zlo=0, zhi=int(math.ceil(0.1 * nz)),
                storage=storage, steps=steps,
                init=dict(kind="noisy_temperature", rho0=0.30, amp=1e-3, T0=0.95 * PR_TC, seed=3))


def pr_droplet(n: int = 384, steps: int = 3000, storage: str = "f32", radius: float = 48.0) -> Case:
    """3-D periodic Peng-Robinson droplet at T/Tc = 0.9 (density ratio ~ 8),
    heat source, no gravity (temperature scale of PR_DROP_SCALE)."""
    s = PR_DROP_SCALE
    return Case(name=f"pr_droplet_{n}", dim=3, nx=n, ny=n, nz=n, eos="pr", R=1.0, cv=2.5,
                Tc=PR_TC * s, Pc=PR_PC * s, omega=PR_OMEGA, kappa=0.2 * s, eta_over_mu=10.0,
                k_over_mu=3.5, q=5e-7 * s, phi_central=1, storage=storage, steps=steps,
                init=dict(kind="droplet", radius=radius, width=2.0, rho_l=2.10988, rho_v=0.26314,
                          T0=0.9 * PR_TC * s, seed=5, amp=0.01, shell=4.0))


def thermal_couette(n: int = 256, nz: int = 128, steps: int = 2000, storage: str = "f32") -> Case:
    """3-D thermal Couette flow (App. B) between non-equilibrium-extrapolation
    walls on z = 0 (at rest, T_C) and z = nz - 1 (moving in x, T_H), ideal gas,
    Pr = 2; linear initial profiles with seeded density noise."""
    return Case(name=f"thermal_couette_{n}x{n}x{nz}", dim=3, nx=n, ny=n, nz=nz, zwalls=2, eos="ideal", R=1.0,
                cv=2.5, k_over_mu=1.75, phi_central=1, uw_hi=(0.1, 0.0, 0.0), Tw_lo=0.33, Tw_hi=0.35,
                storage=storage, steps=steps, init=dict(kind="couette", rho0=3.0, amp=1e-3, seed=12))


def fanno_duct(n: int = 128, nz: int = 256, steps: int = 2000, storage: str = "f32") -> Case:
    """A bundle of n x n periodic-in-xy ducts along z (Sec. III.A, Fanno flow):
    total-state inlet at z = 0, pressure outlet at nz - 1, duct friction,
    ideal gas starting at Ma 0.3 with seeded density noise."""
    T_in, P_in, ma = 0.1, 0.1, 0.3
    gam = 3.5 / 2.5
    T0 = T_in * (1.0 + 0.5 * (gam - 1.0) * ma * ma)
    P0 = P_in * (T0 / T_in) ** 3.5
    return Case(name=f"fanno_duct_{n}x{n}x{nz}", dim=3, nx=n, ny=n, nz=nz, zwalls=2, eos="ideal", R=1.0, cv=2.5,
                k_over_mu=3.5 / 0.71, phi_central=1, friction=4e-3 * 40.0 / nz, face_kind=(1, 3),
                face_P=(P0, 0.08), Tw_lo=T0, Tw_hi=T0, storage=storage, steps=steps,
                init=dict(kind="duct", rho0=P_in / T_in, u0=ma * math.sqrt(gam * T_in), T0=T_in))


def vdw_batch(nsim: int = 64, steps: int = 2000, seed: int = 4, lmin: int = 64, lmax: int = 1024,
              storage: str = "f32") -> list[Case]:
    """Independent 2-D van der Waals quenches: side lengths log-uniform over
    [lmin, lmax], rounded to a multiple of 8 cells (every row of every
    simulation then starts on a 32-byte boundary, so rows are staged by
    16-byte copies), T/Tc uniform over [0.8, 0.98], mean density rho_c."""
    xi = uniform_pm1(seed, 2 * nsim)
    cases = []
    for s in range(nsim):
        L = 8 * int(round(math.exp(math.log(lmin) + (xi[2 * s] + 1.0) * 0.5 * (math.log(lmax) - math.log(lmin))) / 8.0))
        Tr = 0.8 + (xi[2 * s + 1] + 1.0) * 0.5 * 0.18
        c = vdw_spinodal(n=L, steps=steps, storage=storage, Tr=Tr, rho0=VDW_RHOC, seed=1000 + s)
        cases.append(replace(c, name=f"vdw_batch_{s}_{L}"))
    return cases


def window(case: Case, center, half: int, full_z: bool = False):
    """Sub-case over the periodic window [c - half, c + half) of `case` around
    `center` (the full z extent when full_z, e.g. between walls) and its
    initial fields sliced from the case's: a bounded sample of a large
    workload (the window is closed periodically at its faces)."""
    rho, u, T = case.fields()
    shape = (case.nz, case.ny, case.nx)
    ix = (center[0] + np.arange(-half, half)) % case.nx
    iy = (center[1] + np.arange(-half, half)) % case.ny
    iz = np.arange(case.nz) if full_z else (center[2] + np.arange(-half, half)) % case.nz
    sel = np.ix_(iz, iy, ix)
    rw = rho.reshape(shape)[sel].ravel()
    Tw = T.reshape(shape)[sel].ravel()
    uw = np.stack([u[a].reshape(shape)[sel].ravel() for a in range(case.dim)])
    sub = replace(case, name=case.name + "_window", nx=len(ix), ny=len(iy), nz=len(iz))
    return sub, (rw, uw, Tw), sel
