"""The allocation-free step (lbm_step_static) against the handle-based path.

lbm_step_static serves callers that cannot allocate device memory when they
step a simulation: hosts that hand the library a fixed device-memory budget,
programs linking the library without PyTorch's allocator, loops that must
not call cudaMalloc or cudaFree.  Its work arrays sit in a fixed static
device array.  Two calls in a row must reproduce two steps of the regular
entry point (lbm_create/lbm_init/lbm_step, read back with lbm_populations)
to the float64 parity tolerance of the suite, 1e-12 relative.  This file is
collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from paper_2609_28679_b300 import lbm
from paper_2609_28679_b300 import workloads as wl
from tests.util import rel_linf

pytestmark = pytest.mark.gpu


def _cases():
    ideal = wl.acoustic_shear(n=40, storage="f64")
    ideal.ny = 33
    vdw = wl.vdw_spinodal(n=48, ny=37, storage="f64")
    slab = wl.pr_heated_slab(n=12, nz=9, storage="f64")
    slab.ny = 10
    slab.zhi = 3
    return [ideal, vdw, slab]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c.name)
def test_static_step_matches_handle_two_calls(case):
    import torch

    sim = lbm.Simulation(case)
    sim.init()
    f0, g0 = sim.populations()
    sim.step(1)
    f1, g1 = sim.populations()
    sim.step(1)
    f2, g2 = sim.populations()
    sim.close()

    lat, eos, force, heat = lbm.structs_from_case(case)
    stream = torch.cuda.current_stream().cuda_stream
    fa, ga = torch.from_numpy(f0).cuda(), torch.from_numpy(g0).cuda()
    fb, gb = torch.empty_like(fa), torch.empty_like(ga)
    lbm.lbm_step_static(lat, eos, case.tau_f, case.tau_g, force, heat, fa, ga, fb, gb, stream)
    torch.cuda.synchronize()
    assert rel_linf(fb.cpu().numpy(), f1) <= 1e-12
    assert rel_linf(gb.cpu().numpy(), g1) <= 1e-12
    lbm.lbm_step_static(lat, eos, case.tau_f, case.tau_g, force, heat, fb, gb, fa, ga, stream)
    torch.cuda.synchronize()
    assert rel_linf(fa.cpu().numpy(), f2) <= 1e-12
    assert rel_linf(ga.cpu().numpy(), g2) <= 1e-12


def test_static_step_rejects_oversized_lattice():
    import torch

    case = wl.acoustic_shear(n=512, storage="f64")  # 262144 cells > 65536
    lat, eos, force, heat = lbm.structs_from_case(case)
    buf = torch.zeros(9 * 8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError, match="exceed the static maximum"):
        lbm.lbm_step_static(lat, eos, 0.8, 0.8, force, heat, buf, buf.clone(), buf.clone(), buf.clone())


def test_static_step_rejects_what_it_does_not_run():
    import torch

    buf = torch.zeros(27 * 64, dtype=torch.float64, device="cuda")
    # the checks lbm_create makes: Peng-Robinson with b = 0, van der Waals with a < 0
    pr = wl.pr_heated_slab(n=4, nz=4, storage="f64")
    lat, eos, force, heat = lbm.structs_from_case(pr)
    eos.a, eos.b = 0.5, 0.0
    with pytest.raises(lbm.LbmError, match="b > 0"):
        lbm.lbm_step_static(lat, eos, 0.8, 0.8, force, heat, buf, buf.clone(), buf.clone(), buf.clone())
    vdw = wl.vdw_spinodal(n=8, storage="f64")
    lat, eos, force, heat = lbm.structs_from_case(vdw)
    eos.a = -1.0
    with pytest.raises(lbm.LbmError, match="a, b >= 0"):
        lbm.lbm_step_static(lat, eos, 0.8, 0.8, force, heat, buf, buf.clone(), buf.clone(), buf.clone())
    # the learned temperature start needs a handle's parameters
    lat, eos, force, heat = lbm.structs_from_case(pr)
    eos.t_solver = lbm.LBM_T_MLP
    with pytest.raises(lbm.LbmError, match="Newton only"):
        lbm.lbm_step_static(lat, eos, 0.8, 0.8, force, heat, buf, buf.clone(), buf.clone(), buf.clone())
    # outputs overlapping the inputs
    lat, eos, force, heat = lbm.structs_from_case(vdw)
    with pytest.raises(lbm.LbmError, match="alias"):
        lbm.lbm_step_static(lat, eos, 0.8, 0.8, force, heat, buf, buf.clone(), buf[8:], buf.clone())
