"""Linear stability of the oracle's time step about a uniform state (test and
analysis infrastructure; the CUDA path never imports it).

A uniform state (rho, u, T) with no force or source is a fixed point of the
step (Sec. II.E: f* = f^eq when u* = u, theta* = theta and Phi = 0), and the
step commutes with translations along a periodic lattice axis.  Its
Jacobian is then block-circulant: the response R_j[p, m] of population p at
cell m to a unit change of population j at cell 0 gives, for every Fourier
mode exp(i k c) along the axis, the amplification matrix

    A(k)[p, j] = sum_m R_j[p, m] exp(-i k m)          (k = 2 pi s / N)

of one time step (2 Q unknowns per cell: f then g).  The state is linearly
stable when every eigenvalue of every A(k) has modulus <= 1.  R is taken
from the oracle itself by central differences (one perturbed step per
column), so the analysis is of the discrete scheme as built, with every
reading it contains.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as orc


def column_case(case, n: int, axis: int = 2):
    """Params of a periodic 1 x 1 x n column (axis 2) or n x 1 row (axis 0) of
    the case's fluid and relaxation, no force, no source, no walls."""
    dims = [1, 1, 1]
    dims[axis] = n
    p = orc.params_from_case(case)
    p.dim = 3
    p.nx, p.ny, p.nz = dims
    p.zwalls = 0
    p.face_kind[0] = p.face_kind[1] = 0
    p.accel[0] = p.accel[1] = p.accel[2] = 0.0
    p.q = 0.0
    p.zlo = p.zhi = 0
    p.friction = 0.0
    p.throttle_K = 0.0
    return p


def amplification(params, rho: float, u, T: float, h: float = 1e-7):
    """Spectral radius of the one-step amplification matrix A(k) for every
    wavenumber k of the periodic lattice described by params (a column: only
    one of nx, ny, nz above 1), about the uniform state (rho, u, T).
    Returns (k, radius[k], fixed_point_residual)."""
    n = params.nx * params.ny * params.nz
    Q = 27 if params.dim == 3 else 9
    o = orc.Oracle(params)
    dim = params.dim
    o.init(np.full(n, rho), np.tile(np.asarray(u, dtype=np.float64)[:dim, None], (1, n)), np.full(n, T))
    f0, g0 = o.populations()
    Tg = np.full(n, T)
    o.step(1)
    f1, g1 = o.populations()
    resid = max(np.max(np.abs(f1 - f0)) / np.max(np.abs(f0)), np.max(np.abs(g1 - g0)) / np.max(np.abs(g0)))
    x0 = np.concatenate([f0, g0])  # [2Q][n]
    R = np.zeros((2 * Q, 2 * Q, n))  # R[j][p, m]
    for j in range(2 * Q):
        scale = max(abs(x0[j, 0]), 1e-3 * np.max(np.abs(x0[j // Q * Q:(j // Q + 1) * Q])))
        resp = []
        for sgn in (1.0, -1.0):
            x = x0.copy()
            x[j, 0] += sgn * h * scale
            o.set_populations(x[:Q], x[Q:], Tg)
            o.step(1)
            f, g = o.populations()
            resp.append(np.concatenate([f, g]))
        R[j] = (resp[0] - resp[1]) / (2.0 * h * scale)
    k = 2.0 * np.pi * np.arange(n) / n
    phase = np.exp(-1j * np.outer(k, np.arange(n)))  # [k][m]
    radius = np.zeros(n)
    for s in range(n):
        A = np.einsum("jpm,m->pj", R, phase[s])
        radius[s] = np.max(np.abs(np.linalg.eigvals(A)))
    return k, radius, resid
