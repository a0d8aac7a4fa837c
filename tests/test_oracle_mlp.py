"""Pins of the FP64 MLP reference: backprop against central finite
differences, and a small Adam fit of the Peng-Robinson inversion (samples
from the oracle's EoS and Newton solver) that must beat the constant guess."""
import numpy as np
import pytest

from oracle import mlp
from oracle import oracle as orc
from paper_2609_28679_b300 import workloads as wl


def _pr_eos():
    c = wl.pr_droplet(n=8)
    a, b = orc.pr_from_critical(c.R, c.Tc, c.Pc)
    return orc.EoS(orc.make_params(eos="pr", R=c.R, cv=c.cv, a=a, b=b, Tc=c.Tc, omega=c.omega)), c.Tc


def _samples(n, seed):
    eos, Tc = _pr_eos()
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(np.log(0.1), np.log(2.6), n))
    T = rng.uniform(0.85, 1.05, n) * Tc
    e = np.array([eos.e(r, t) for r, t in zip(rho, T)])
    Tn = np.array([eos.T(r, ee, 0.0)[0] for r, ee in zip(rho, e)])  # Newton from Tc
    return rho, e, Tn, Tc


def test_backprop_matches_finite_differences():
    rho, e, T, Tc = _samples(20, 1)
    p = mlp.init_params((0.1, 2.6), (e.min(), e.max()), (0.85 * Tc, 1.05 * Tc), seed=3)
    p[mlp.N_NORM:] += np.random.default_rng(4).normal(0, 0.05, mlp.N_PARAMS - mlp.N_NORM)
    loss, g = mlp.loss_and_grad(p, rho, e, T)
    rng = np.random.default_rng(5)
    idx = np.concatenate([np.arange(mlp.N_NORM, mlp.N_NORM + 40), rng.integers(mlp.N_NORM, mlp.N_PARAMS, 80),
                          [mlp.N_PARAMS - 1]])
    h = 1e-5  # central differences: truncation O(h^2), rounding eps*L/h
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss_and_grad(pp, rho, e, T)[0] - mlp.loss_and_grad(pm, rho, e, T)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-12)
    assert np.all(g[:mlp.N_NORM] == 0)


def test_adam_fit_learns_the_inversion():
    rho, e, T, Tc = _samples(2000, 2)
    p0 = mlp.init_params((0.1, 2.6), (e.min(), e.max()), (0.85 * Tc, 1.05 * Tc), seed=1)
    l0, _ = mlp.loss_and_grad(p0, rho, e, T)
    p = mlp.adam_train(p0, rho, e, T, epochs=30, batch=100, lr=3e-3)
    l1, _ = mlp.loss_and_grad(p, rho, e, T)
    That, _ = mlp.forward(p, rho, e)
    assert l1 < 0.02 * l0
    assert np.max(np.abs(That - T)) / Tc < 0.05


def test_bf16_rounding_is_nearest_ties_to_even():
    # 7 fraction bits: the spacing at 1 is 2^-7; halfway cases go to the even neighbour
    cases = [(1.0, 1.0), (1 + 2 ** -9, 1.0), (1 + 2 ** -8, 1.0), (1 + 3 * 2 ** -9, 1 + 2 ** -7),
             (1 + 2 ** -7 + 2 ** -8, 1 + 2 ** -6), (-2.5, -2.5), (3 + 2 ** -7, 3.0), (65280.0, 65280.0),
             (-(1 + 3 * 2 ** -9), -(1 + 2 ** -7))]
    for x, r in cases:
        assert mlp.bf16(x) == r, (x, mlp.bf16(x), r)
    # every rounded value is a float32 whose lower 16 bits are zero, within half a spacing of the input
    x = np.random.default_rng(6).normal(0, 3, 1000)
    r = mlp.bf16(x)
    assert np.all((r.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)
    assert np.all(np.abs(r - x.astype(np.float32)) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))


def test_bf16_product_gradient():
    # The rounded computation is smooth in b2, W3 and b3 (they act after the
    # rounded product): its gradient there must match central differences of
    # its own loss.  Through the rounded operands it stays within the rounding
    # (a few 2^-9 relative) of the exact gradient.
    rho, e, T, Tc = _samples(40, 7)
    p = mlp.init_params((0.1, 2.6), (e.min(), e.max()), (0.85 * Tc, 1.05 * Tc), seed=8)
    p[mlp.N_NORM:] += np.random.default_rng(9).normal(0, 0.1, mlp.N_PARAMS - mlp.N_NORM)
    _, gb = mlp.loss_and_grad(p, rho, e, T, bf16_products=True)
    _, gx = mlp.loss_and_grad(p, rho, e, T)
    o = mlp.N_NORM + 2 * mlp.H + mlp.H + mlp.H * mlp.H  # first b2 entry
    h = 1e-5
    for k in list(range(o, o + 2 * mlp.H + 1, 7)) + [mlp.N_PARAMS - 1]:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss_and_grad(pp, rho, e, T, bf16_products=True)[0] -
              mlp.loss_and_grad(pm, rho, e, T, bf16_products=True)[0]) / (2 * h)
        assert gb[k] == pytest.approx(fd, rel=1e-6, abs=1e-12)
    db, dx = mlp.unpack(gb), mlp.unpack(gx)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.linalg.norm(db[name] - dx[name]) / np.linalg.norm(dx[name])
        assert 0 < err <= 2e-2, (name, err)
