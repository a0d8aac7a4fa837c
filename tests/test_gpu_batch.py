"""Batched form: many independent simulations in one fused launch per step
(uneven sizes, per-simulation parameters), CUDA-graph replay of step chunks,
and the autotuner (chooses a kernel, leaves the state untouched)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_28679_b300 import lbm
from paper_2609_28679_b300 import workloads as wl
from tests.util import oracle_params, rel_linf

pytestmark = pytest.mark.gpu


def test_batched_fused_matches_oracle_per_simulation():
    cases = wl.vdw_batch(nsim=5, lmin=12, lmax=45, storage="f64", steps=8)
    sim = lbm.Simulation(cases, variant=lbm.LBM_KERNEL_FUSED)
    assert sim.kernel()[0] == lbm.LBM_KERNEL_FUSED
    sim.init()
    sim.step(8)
    rho, u, T = sim.moments()
    inv = sim.invariants()
    off = 0
    for s, c in enumerate(cases):
        o = orc.Oracle(oracle_params(c))
        o.init(*c.fields())
        o.step(8)
        rr, ur, Tr = o.moments()
        n = c.ncell
        assert rel_linf(rho[off:off + n], rr) <= 1e-12
        assert rel_linf(T[off:off + n], Tr) <= 1e-12
        assert np.max(np.abs(u[2 * off:2 * off + 2 * n] - ur.ravel())) <= 1e-12 * max(np.abs(ur).max(), 1e-3)
        oi = o.invariants()
        assert abs(inv[s][0] - oi[0]) <= 1e-12 * oi[0]
        off += n


def test_row_march_graph_replay_matches_eager_steps():
    # the 2-D row march (float32) under graph replay: the same launches, bit for bit
    import torch

    c = wl.vdw_spinodal(n=136, ny=44, storage="f32")
    eager = lbm.Simulation(c, variant=lbm.LBM_KERNEL_YMARCH)
    assert eager.kernel()[0] == lbm.LBM_KERNEL_YMARCH
    eager.init()
    eager.step(18)
    stream = torch.cuda.Stream()
    g = lbm.Simulation(c, variant=lbm.LBM_KERNEL_YMARCH)
    g.use_graphs(4, stream)
    g.init()
    g.step(13)
    g.step(5)
    fe, ge = eager.populations()
    fg, gg = g.populations()
    assert np.array_equal(fg, fe)
    assert np.array_equal(gg, ge)


@pytest.mark.parametrize("variant", [lbm.LBM_KERNEL_SPLIT, lbm.LBM_KERNEL_FUSED])
def test_graph_replay_matches_eager_steps(variant):
    import torch

    c = wl.vdw_spinodal(n=40, ny=28, storage="f64")
    eager = lbm.Simulation(c, variant=variant)
    eager.init()
    eager.step(13)
    fe, ge = eager.populations()
    stream = torch.cuda.Stream()
    g = lbm.Simulation(c, variant=variant)
    g.use_graphs(4, stream)
    g.init()
    g.step(13)   # 1 eager + 3 graphs of 4
    g.step(5)    # parity changed: graph of the other parity
    g.step(0)
    eager.step(5)
    fe, ge = eager.populations()
    fg, gg = g.populations()
    assert rel_linf(fg, fe) <= 1e-13
    assert rel_linf(gg, ge) <= 1e-13


def test_autotune_picks_a_kernel_and_restores_the_state():
    c = wl.vdw_spinodal(n=96, storage="f32")
    sim = lbm.Simulation(c)
    sim.init()
    sim.step(3)
    f0, g0 = sim.populations()
    d0 = sim.diagnostics()
    (variant, tx, ty, tz), ms = sim.autotune(3)
    assert variant in (lbm.LBM_KERNEL_SPLIT, lbm.LBM_KERNEL_FUSED) and ms > 0
    assert sim.kernel() == (variant, tx, ty, tz)
    f1, g1 = sim.populations()
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    assert np.array_equal(d0, sim.diagnostics())
    ref = lbm.Simulation(c, variant=lbm.LBM_KERNEL_SPLIT)
    ref.init()
    ref.step(5)
    sim.step(2)
    assert rel_linf(sim.moments()[0], ref.moments()[0]) <= 1e-5
