"""Parity at the full sizes of the five workload configurations, in the launch
configuration bench.py times (the autotuned kernel and tile).

The 2-D workloads (128^2, 512^2, the 64-simulation batch) are compared with a
full oracle run, element by element.  The 3-D ones (256^3, 384^3) are
compared on sampled cells: the oracle steps a window of the initial fields
(periodic closure at the window's faces, the real walls kept in z) and the
cells farther from the faces than the dependency radius of the steps taken
evolve exactly as in the full domain.  One step reaches 5 cells (the
Korteweg force needs rho two cells out, the upwind Phi the state two cells
out of that, streaming one more); the margins below are 6 per step.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_28679_b300 import lbm
from paper_2609_28679_b300 import workloads as wl
from tests.util import oracle_params, rel_linf

pytestmark = pytest.mark.gpu

RADIUS = 6  # cells per step (see module docstring)


def _gpu_run(case, steps, fields=None, mlp=None):
    sim = lbm.Simulation(case)
    if mlp is not None:
        lbm.lbm_mlp_load(sim.h, mlp)
    sim.init(fields)
    sim.autotune(3)  # bench.py's launch configuration; the state is restored
    sim.step(steps)
    rho, u, T = sim.moments()
    kernel = sim.kernel()
    sim.close()
    return (rho, u, T), kernel


def _check(got, ref, tol, what=""):
    rho, u, T = got
    rr, ur, Tr = ref
    assert rel_linf(rho, rr) <= tol, what
    assert rel_linf(T, Tr) <= tol, what
    du = float(np.max(np.abs(np.asarray(u).ravel() - np.asarray(ur).ravel())))
    assert du <= tol, (what, du)


def _full_oracle(case, steps, fields=None):
    o = orc.Oracle(oracle_params(case))
    o.init(*(fields if fields is not None else case.fields()))
    o.step(steps)
    return o.moments()


def test_cfg1_acoustic_shear_128_f64():
    c = wl.acoustic_shear(128, storage="f64")
    got, _ = _gpu_run(c, 50)
    _check(got, _full_oracle(c, 50), 1e-12)


def test_cfg2_vdw_512_f32_bench_kernel():
    c = wl.vdw_spinodal(512, storage="f32")
    got, kernel = _gpu_run(c, 10)
    assert kernel[0] == lbm.LBM_KERNEL_FUSED  # the variant the bench line times
    _check(got, _full_oracle(c, 10), 1e-5)


def test_cfg4_batch_64_f32():
    cases = wl.vdw_batch(64, storage="f32")
    sim = lbm.Simulation(cases)
    sim.init()
    sim.autotune(3)
    sim.step(5)
    rho, u, T = sim.moments()
    sim.close()
    off = 0
    for c in cases:
        n = c.ncell
        ref = _full_oracle(c, 5)
        got = (rho[off:off + n], u[:, off:off + n] if u.ndim == 2 else u[2 * off:2 * (off + n)], T[off:off + n])
        _check(got, ref, 1e-5, c.name)
        off += n


def _window(case, center, half, walls_z):
    """Sub-case and initial fields of the window [c - half, c + half) around
    center (periodic indices); full extent in z when the case has walls."""
    rho, u, T = case.fields()
    nx, ny, nz = case.nx, case.ny, case.nz
    shape = (nz, ny, nx)
    ix = (center[0] + np.arange(-half, half)) % nx
    iy = (center[1] + np.arange(-half, half)) % ny
    iz = np.arange(nz) if walls_z else (center[2] + np.arange(-half, half)) % nz
    sel = np.ix_(iz, iy, ix)
    rw = rho.reshape(shape)[sel].ravel()
    Tw = T.reshape(shape)[sel].ravel()
    uw = np.stack([u[a].reshape(shape)[sel].ravel() for a in range(3)])
    sub = wl.Case(**{**case.__dict__, "name": case.name + "_window", "nx": len(ix), "ny": len(iy), "nz": len(iz)})
    return sub, (rw, uw, Tw), sel


def _window_check(case, center, half, steps, got, tol):
    walls = bool(case.zwalls)
    sub, fields, sel = _window(case, center, half, walls)
    o = orc.Oracle(oracle_params(sub))
    o.init(*fields)
    o.step(steps)
    rr, ur, Tr = o.moments()
    shape_w = (sub.nz, sub.ny, sub.nx)
    m = RADIUS * steps
    inner = (slice(None) if walls else slice(m, -m), slice(m, -m), slice(m, -m))
    shape = (case.nz, case.ny, case.nx)
    rho, u, T = got
    g_rho = rho.reshape(shape)[sel][inner]
    g_T = T.reshape(shape)[sel][inner]
    g_u = np.stack([u[a].reshape(shape)[sel][inner] for a in range(3)])
    o_rho = rr.reshape(shape_w)[inner]
    o_T = Tr.reshape(shape_w)[inner]
    o_u = np.stack([ur[a].reshape(shape_w)[inner] for a in range(3)])
    assert g_rho.size > 1000
    _check((g_rho, g_u, g_T), (o_rho, o_u, o_T), tol, case.name)


# float32 with the central Phi: the upwind-biased derivative takes its branch
# from the sign of u, and where u rounds across zero float32 and the float64
# oracle take different (equally valid) branches; that deviation is measured
# and bounded by the test below instead of being compared element by element.
@pytest.mark.parametrize("storage,tol,central", [("f32", 1e-5, 1), ("bf16", 2e-3, 0), ("f16", 3e-4, 0)])
def test_cfg3_pr_slab_256_sampled(storage, tol, central):
    c = wl.pr_heated_slab(256, storage=storage)
    c.phi_central = central
    got, kernel = _gpu_run(c, 2)
    u = got[1].reshape(3, -1)
    got = (got[0], u, got[2])
    # a column through the heated layer and the walls, away from the x/y origin
    _window_check(c, (131, 77, 0), 20, 2, got, tol)


def test_cfg3_pr_slab_256_f32_upwind_deviation():
    # The workload as configured (upwind-biased Phi) at float32: the branch
    # flips where u rounds across zero are the only source beyond float32
    # rounding (central Phi: 8e-7 on the same window).  Measured on a B300:
    # 0.6-1.1e-5 in rho after 2 steps for every kernel; bounded at 5e-5.
    c = wl.pr_heated_slab(256, storage="f32")
    got, kernel = _gpu_run(c, 2)
    u = got[1].reshape(3, -1)
    got = (got[0], u, got[2])
    _window_check(c, (131, 77, 0), 20, 2, got, 5e-5)


def _trained_params(case):
    le = lbm.structs_from_case(case)[1]
    params = np.zeros(lbm.lbm_mlp_nparams(), dtype=np.float32)
    lbm.lbm_mlp_train(le, (0.1, 2.6, 0.85, 1.05), 1 << 16, 1500, 512, 2e-3, 7, True, params)
    return params


@pytest.mark.parametrize("learned", [False, True])
def test_cfg5_pr_droplet_384_sampled(learned):
    c = wl.pr_droplet(384, storage="f32")
    mlp = None
    if learned:
        c.t_solver = 1
        mlp = _trained_params(c)
    got, _ = _gpu_run(c, 1, mlp=mlp)
    u = got[1].reshape(3, -1)
    got = (got[0], u, got[2])
    # centred on the droplet's interface (radius 48 about the domain centre)
    _window_check(c, (192 + 48, 192, 192), 18, 1, got, 1e-5)
