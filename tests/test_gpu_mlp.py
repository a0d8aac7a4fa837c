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


_TRAINED = {}


def _trained_params():
    if "p" not in _TRAINED:
        c, _ = _pr()
        le = lbm.structs_from_case(c)[1]
        params = np.zeros(lbm.lbm_mlp_nparams(), dtype=np.float32)
        lbm.lbm_mlp_train(le, (0.1, 2.6, 0.85, 1.05), 1 << 16, 1500, 512, 2e-3, 7, True, params)
        _TRAINED["p"] = params
    return _TRAINED["p"]


def test_learned_start_keeps_f64_parity_with_oracle():
    # the network only seeds Newton; the float64 path converges to 1e-14 either way
    c = wl.pr_droplet(n=14, radius=4.0, storage="f64")
    c.t_solver = 1
    sim = lbm.Simulation(c)
    lbm.lbm_mlp_load(sim.h, _trained_params())
    sim.init()
    sim.step(6)
    rho, u, T = sim.moments()
    o = orc.Oracle(orc.params_from_case(c))
    o.init(*c.fields())
    o.step(6)
    rr, ur, Tr = o.moments()
    assert np.max(np.abs(rho - rr)) / rr.max() <= 1e-12
    assert np.max(np.abs(T - Tr)) / Tr.max() <= 1e-12


@pytest.mark.parametrize("variant", [lbm.LBM_KERNEL_SPLIT, lbm.LBM_KERNEL_FUSED])
def test_learned_start_f32_matches_newton_run(variant):
    # float32 Newton stops at |dT| <= 1e-6 T from either start; the runs agree to that level
    base = wl.pr_droplet(n=16, radius=5.0, storage="f32")
    newton = lbm.Simulation(base, variant=variant)
    newton.init()
    newton.step(10)
    c = wl.pr_droplet(n=16, radius=5.0, storage="f32")
    c.t_solver = 1
    sim = lbm.Simulation(c)
    lbm.lbm_mlp_load(sim.h, _trained_params())
    lbm.lbm_set_kernel(sim.h, variant)
    assert sim.kernel()[0] == variant
    sim.init()
    sim.step(10)
    r1, u1, T1 = sim.moments()
    r0, u0, T0 = newton.moments()
    assert np.max(np.abs(r1 - r0)) / r0.max() <= 1e-5
    assert np.max(np.abs(T1 - T0)) / T0.max() <= 1e-5
    d = sim.diagnostics()
    assert d[0] == 0
    assert 0 <= d[3] <= 10 * c.ncell


def test_learned_start_saves_newton_iterations_over_a_cold_start():
    # What the trained network gains: float64 Newton iterations (oracle solver) to
    # converge from T_hat versus from Tc, the start without a previous T.
    c, eos = _pr()
    rho, e, T, _ = _samples(400, 21)
    That = lbm.lbm_mlp_predict(_trained_params(), rho, e)
    it_cold = np.array([eos.T(r, ee, 0.0)[1] for r, ee in zip(rho, e)])
    it_mlp = np.array([eos.T(r, ee, t0)[1] for r, ee, t0 in zip(rho, e, That)])
    assert np.mean(it_mlp) < np.mean(it_cold)
    assert np.max(it_mlp) <= np.max(it_cold)
