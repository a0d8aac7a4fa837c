"""Pins of the oracle's lattice and equilibria (Sec. II.C) against facts that do
not come from the oracle itself: textbook lattice weights, exact moment
identities of the product form, and symbolic application of the
generating-function operators of Eq. LBMeqG."""
import itertools

import numpy as np
import pytest
import sympy as sp

from oracle import oracle as orc

RNG = np.random.default_rng(12345)


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_is_full_tensor_product(dim):
    c, opp = orc.lattice(dim)
    Q = 3 ** dim
    assert c.shape == (Q, dim)
    assert len({tuple(v) for v in c}) == Q            # every velocity in {-1,0,1}^D once
    assert np.all(c[opp] == -c)                        # opposite directions
    assert np.all(c.sum(axis=0) == 0)


def test_d2q9_rest_weights_textbook():
    # theta = varsigma^2 = 1/3 at rest gives the standard D2Q9 weights 4/9, 1/9, 1/36.
    c, _ = orc.lattice(2)
    f = orc.feq(2, 1.0, [0.0, 0.0], 1.0 / 3.0)
    n2 = (c ** 2).sum(axis=1)
    expected = np.select([n2 == 0, n2 == 1, n2 == 2], [4 / 9, 1 / 9, 1 / 36])
    np.testing.assert_allclose(f, expected, rtol=0, atol=4e-16)


def test_d3q27_rest_weights_textbook():
    c, _ = orc.lattice(3)
    f = orc.feq(3, 1.0, [0.0, 0.0, 0.0], 1.0 / 3.0)
    n2 = (c ** 2).sum(axis=1)
    expected = np.select([n2 == 0, n2 == 1, n2 == 2, n2 == 3], [8 / 27, 2 / 27, 1 / 54, 1 / 216])
    np.testing.assert_allclose(f, expected, rtol=0, atol=4e-16)


def test_psi_special_values():
    # Eq. phi: Psi = 1 - zeta at c = 0 and (zeta +- xi)/2 at c = +-1.
    xi, zeta = 0.37, 0.29
    assert orc.psi(0, xi, zeta) == pytest.approx(1 - zeta, abs=1e-16)
    assert orc.psi(1, xi, zeta) == pytest.approx((zeta + xi) / 2, abs=1e-16)
    assert orc.psi(-1, xi, zeta) == pytest.approx((zeta - xi) / 2, abs=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_feq_moments(dim):
    # Eq. LBMeq: zeroth, first and second moments of the product form are exact.
    c, _ = orc.lattice(dim)
    for _ in range(20):
        rho = RNG.uniform(0.2, 5.0)
        u = RNG.uniform(-0.3, 0.3, dim)
        th = RNG.uniform(0.1, 0.6)
        f = orc.feq(dim, rho, u, th)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(c.T @ f, rho * u, rtol=0, atol=1e-14 * rho)
        P2 = (c[:, :, None] * c[:, None, :] * f[:, None, None]).sum(axis=0)
        np.testing.assert_allclose(P2, rho * (th * np.eye(dim) + np.outer(u, u)), rtol=0, atol=1e-14 * rho)
        # diagonal third moment is rho u_alpha (c^3 = c): the lattice defect Phi corrects
        np.testing.assert_allclose((c ** 3).T @ f, rho * u, rtol=0, atol=1e-14 * rho)


@pytest.mark.parametrize("dim", [2, 3])
def test_fstar_moments(dim):
    # Eq. LBMstar: sum f* = rho, sum c f* = rho u*, diag second moment = rho(theta* + u*^2 + Phi).
    c, _ = orc.lattice(dim)
    rho, us, ths = 1.7, RNG.uniform(-0.2, 0.2, dim), 0.41
    Phi = RNG.uniform(-0.05, 0.05, dim)
    f = orc.fprod(dim, rho, us, ths + us * us + Phi)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    np.testing.assert_allclose(c.T @ f, rho * us, atol=1e-14)
    np.testing.assert_allclose((c ** 2).T @ f, rho * (ths + us * us + Phi), atol=1e-14)


def _geq_symbolic(dim):
    """g_i = rho prod_alpha Psi(c_ia; O_a, O_a^2) E with O_a = theta d/du_a + u_a (Eqs. Oa, LBMeqG),
    applied literally to E = e + |u|^2/2 with sympy."""
    u = sp.symbols(f"u0:{dim}")
    th, e, rho = sp.symbols("theta e rho")
    E = e + sum(ui ** 2 for ui in u) / 2

    def O(expr, a):
        return th * sp.diff(expr, u[a]) + u[a] * expr

    def Psi_op(expr, a, c):
        o1 = O(expr, a)
        o2 = O(o1, a)
        return (1 - c * c) * expr + sp.Rational(1, 2) * ((3 * c * c - 2) * o2 + c * o1)

    out = []
    for digits in itertools.product([0, 1, 2], repeat=dim):
        # direction index i = d0 + 3 d1 + 9 d2, digit -> c = 0, +1, -1
        cs = [0 if d == 0 else (1 if d == 1 else -1) for d in digits]
        expr = E
        for a in range(dim):
            expr = Psi_op(expr, a, cs[a])
        idx = sum(d * 3 ** k for k, d in enumerate(digits))
        out.append((idx, sp.lambdify((rho, u, e, th), sp.expand(rho * expr))))
    out.sort(key=lambda t: t[0])
    return [fn for _, fn in out]


@pytest.mark.parametrize("dim", [2, 3])
def test_geq_matches_operator_form(dim):
    fns = _geq_symbolic(dim)
    for _ in range(5):
        rho = RNG.uniform(0.2, 4.0)
        u = RNG.uniform(-0.4, 0.4, dim)
        e = RNG.uniform(-1.0, 3.0)
        th = RNG.uniform(0.05, 0.7)
        sym = np.array([fn(rho, tuple(u), e, th) for fn in fns])
        num = orc.geq(dim, rho, u, e, th)
        np.testing.assert_allclose(num, sym, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_geq_moments(dim):
    # Sum g^eq = rho E; sum c g^eq = u (rho E + P); diag sum c^2 g^eq = u^2 (rho E + 2P) + (E + P/rho) P,
    # with theta = P/rho (Eqs. gcons_app and the Pi_1, Pi_2 of the g equilibrium in App. A).
    c, _ = orc.lattice(dim)
    rho, u, e, P = 2.3, RNG.uniform(-0.3, 0.3, dim), 1.1, 0.8
    th = P / rho
    E = e + 0.5 * u @ u
    g = orc.geq(dim, rho, u, e, th)
    assert g.sum() == pytest.approx(rho * E, rel=1e-14)
    np.testing.assert_allclose(c.T @ g, u * (rho * E + P), atol=1e-13)
    np.testing.assert_allclose((c ** 2).T @ g, u * u * (rho * E + 2 * P) + (E + P / rho) * P, atol=1e-13)
