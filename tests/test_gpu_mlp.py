"""Learned temperature inversion: the tensor-core training kernel's
gradients and the in-step inference routine against the FP64 oracle of the
same network, and GPU training of the Peng-Robinson inversion.

Tolerances: bfloat16 operands (8-bit mantissa, relative rounding 2^-9) in
the 64-wide layer with float32 accumulation; gradients are compared per
parameter block in the 2-norm relative to the oracle's, at 2e-2; the
network output y (unit scale) to 2e-2 absolute."""
import numpy as np
import pytest

from oracle import mlp
from oracle import oracle as orc
from paper_2609_28679_b300 import lbm
from paper_2609_28679_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _pr():
    c = wl.pr_droplet(n=8)
    a, b = orc.pr_from_critical(c.R, c.Tc, c.Pc)
    return c, orc.EoS(orc.make_params(eos="pr", R=c.R, cv=c.cv, a=a, b=b, Tc=c.Tc, omega=c.omega))


def _samples(n, seed):
    c, eos = _pr()
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(np.log(0.1), np.log(2.6), n))
    T = rng.uniform(0.85, 1.05, n) * c.Tc
    e = np.array([eos.e(r, t) for r, t in zip(rho, T)])
    return rho, e, T, c


def _params(e, Tc, seed):
    p = mlp.init_params((0.1, 2.6), (e.min(), e.max()), (0.85 * Tc, 1.05 * Tc), seed=seed)
    p[mlp.N_NORM:] += np.random.default_rng(seed + 1).normal(0, 0.1, mlp.N_PARAMS - mlp.N_NORM)
    return p.astype(np.float32)


def test_gradients_match_oracle():
    rho, e, T, c = _samples(200, 11)
    p32 = _params(e, c.Tc, 3)
    loss_g, g = lbm.lbm_mlp_grad(p32, rho, e, T)
    loss_r, gr = mlp.loss_and_grad(p32.astype(np.float64), rho, e, T)
    assert loss_g == pytest.approx(loss_r, rel=2e-2)
    d = mlp.unpack(gr)
    dg = mlp.unpack(g.astype(np.float64))
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.linalg.norm(dg[name] - d[name]) / np.linalg.norm(d[name])
        assert err <= 2e-2, (name, err)


def test_inference_matches_oracle_forward():
    rho, e, T, c = _samples(1000, 12)
    p32 = _params(e, c.Tc, 5)
    Tg = lbm.lbm_mlp_predict(p32, rho, e)
    Tr, _ = mlp.forward(p32.astype(np.float64), rho, e)
    s_T = float(p32[5])
    assert np.max(np.abs(Tg - Tr)) / s_T <= 2e-2


def test_training_learns_the_inversion():
    c, eos = _pr()
    le = lbm.structs_from_case(c)[1]
    params = np.zeros(lbm.lbm_mlp_nparams(), dtype=np.float32)
    hist = np.zeros(1500)
    lbm.lbm_mlp_train(le, (0.1, 2.6, 0.85, 1.05), 1 << 16, 1500, 512, 2e-3, 7, True, params, hist)
    assert np.mean(hist[-50:]) < 0.02 * np.mean(hist[:10])
    rho, e, T, _ = _samples(2000, 13)
    Tg = lbm.lbm_mlp_predict(params, rho, e)
    assert np.max(np.abs(Tg - T)) / c.Tc < 0.02
