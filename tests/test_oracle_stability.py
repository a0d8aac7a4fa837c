"""Linear stability of the oracle's time step about uniform flow (reading A5
of the upwind-biased derivative in Eq. correction, and the window of the
supersonic duct cases).  The amplification matrices come from the oracle by
finite differences (oracle/stability.py); the tool itself is pinned by the
closed-form decay rate of a shear wave at rest (Sec. II.D: nu = tau theta)."""
import math

import numpy as np
import pytest

from oracle import stability as st
from paper_2609_28679_b300 import workloads as wl

UPWIND_BIASED, CENTRAL, ONE_SIDED = 0, 1, 2


def _radius(scheme, theta, Ma, tau=0.8, n=16):
    c = wl.fanno_duct(1, 16)
    c.phi_central, c.tau_f, c.tau_g, c.eta_over_mu = scheme, tau, tau, 0.0
    k, r, res = st.amplification(st.column_case(c, n), 1.0, (0.0, 0.0, Ma * math.sqrt(1.4 * theta)), theta)
    assert res <= 1e-14  # uniform flow is a fixed point of the step
    return k, r


def test_shear_wave_rate_pins_the_amplification_matrices():
    # At rest the two shear waves of the smallest wavenumber along the column (u_x and u_y
    # varying along it) are a degenerate pair of real eigenvalues with decay 1 - lambda =
    # nu k^2 to O(k^4), nu = tau theta (Sec. II.D; the lattice's O(k^2) correction is ~1 %).
    theta, tau, n = 0.1, 0.8, 32
    c = wl.fanno_duct(1, 16)
    c.phi_central, c.tau_f, c.tau_g = CENTRAL, tau, tau
    p = st.column_case(c, n)
    k1 = 2 * math.pi / n
    _, o_r, _ = st.amplification(p, 1.0, (0.0, 0.0, 0.0), theta)
    lam = _spectrum(p, theta, 1)
    real = np.sort(lam[np.abs(lam.imag) <= 1e-6].real)
    pairs = [a for a, b in zip(real[:-1], real[1:]) if abs(a - b) <= 1e-7 and a > 0.9]
    decay = 1.0 - math.exp(-tau * theta * k1 ** 2)
    assert any(abs((1.0 - a) - decay) <= 0.02 * decay for a in pairs), (pairs, decay)
    assert o_r[0] == pytest.approx(1.0, abs=1e-6)  # k = 0: conserved mass, momentum, energy


def _spectrum(p, theta, s):
    """All eigenvalues of A(k_s) (same construction as stability.amplification)."""
    from oracle import oracle as orc
    n = p.nx * p.ny * p.nz
    Q = 27
    o = orc.Oracle(p)
    o.init(np.full(n, 1.0), np.zeros((3, n)), np.full(n, theta))
    f0, g0 = o.populations()
    x0 = np.concatenate([f0, g0])
    R = np.zeros((2 * Q, 2 * Q, n))
    h = 1e-7
    for j in range(2 * Q):
        scale = max(abs(x0[j, 0]), 1e-3 * np.max(np.abs(x0[j // Q * Q:(j // Q + 1) * Q])))
        resp = []
        for sgn in (1.0, -1.0):
            x = x0.copy()
            x[j, 0] += sgn * h * scale
            o.set_populations(x[:Q], x[Q:], np.full(n, theta))
            o.step(1)
            f, g = o.populations()
            resp.append(np.concatenate([f, g]))
        R[j] = (resp[0] - resp[1]) / (2 * h * scale)
    ph = np.exp(-1j * 2 * np.pi * s / n * np.arange(n))
    return np.linalg.eigvals(np.einsum("jpm,m->pj", R, ph))


@pytest.mark.parametrize("theta", [0.02, 0.1])
def test_subsonic_uniform_flow_is_stable_with_the_upwind_biased_and_central_phi(theta):
    for scheme in (UPWIND_BIASED, CENTRAL):
        _, r = _radius(scheme, theta, 0.5)
        assert np.max(r) <= 1 + 1e-6, (scheme, np.max(r))  # finite-difference noise ~1e-8


def test_upwind_biased_phi_extends_stability_to_higher_mach_numbers():
    # Sec. II.E: the upwind-biased derivative is there for stability at higher Mach numbers.
    # At Ma 1.2 (theta 0.1) the third-order upwind-biased difference keeps uniform flow stable;
    # the central difference and the fully one-sided second-order difference do not.
    _, r_ub = _radius(UPWIND_BIASED, 0.1, 1.2)
    _, r_c = _radius(CENTRAL, 0.1, 1.2)
    _, r_os = _radius(ONE_SIDED, 0.1, 1.2)
    assert np.max(r_ub) <= 1 + 1e-6
    assert np.max(r_c) > 1.02
    assert np.max(r_os) > 1.2
    # the one-sided difference fails already at Ma 0.5
    _, r_os05 = _radius(ONE_SIDED, 0.1, 0.5)
    assert np.max(r_os05) > 1.2


def test_ma_1_5_window_of_the_supersonic_ducts():
    # at Ma 1.5 uniform flow grows at most weakly with the upwind-biased Phi at theta 0.02,
    # tau 1 (carried out of a finite duct before it matters), strongly with the central Phi
    _, r_ub = _radius(UPWIND_BIASED, 0.02, 1.5, tau=1.0)
    _, r_c = _radius(CENTRAL, 0.02, 1.5, tau=1.0)
    assert np.max(r_ub) <= 1.02
    assert np.max(r_c) > np.max(r_ub)
