"""Per-cell body force F_B(x) and heat source Q(x) given by the caller in
device memory (lbm_force.field, lbm_heat.field; the generic F_B and Q of
Eq. force_decomposition and the energy equation) on the split kernels,
through the C ABI, against the FP64 CPU oracle: element by element in 2-D and
3-D, float64 1e-12 and float32 1e-5, a field changed between steps, and the
kernel rules."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_28679_b300 import lbm
from paper_2609_28679_b300 import workloads as wl
from tests.util import oracle_params, rel_linf

pytestmark = pytest.mark.gpu


def _fields(c, seed, fscale=2e-5, qscale=2e-6):
    rng = np.random.default_rng(seed)
    return fscale * rng.standard_normal((c.dim, c.ncell)), qscale * (1.0 + rng.random(c.ncell))


class _Run:
    """A handle whose force and heat carry per-cell device fields."""

    def __init__(self, c, F, Q):
        import torch

        self.c = c
        self.F = torch.from_numpy(np.ascontiguousarray(F)).cuda()
        self.Q = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
        lat, eos, force, heat = lbm.structs_from_case(c)
        force.field = ctypes.c_void_p(self.F.data_ptr())
        heat.field = ctypes.c_void_p(self.Q.data_ptr())
        self.h = lbm.lbm_create(lat, eos, c.tau_f, c.tau_g, force, heat)
        rho, u, T = c.fields()
        lbm.lbm_init(self.h, rho, np.ascontiguousarray(u).ravel(), T, 0)

    def step(self, n):
        lbm.lbm_step(self.h, n)

    def compare(self, o, tol, f32=False):
        import torch

        torch.cuda.synchronize()
        Qn = 3 ** self.c.dim
        f = np.zeros(Qn * self.c.ncell)
        g = np.zeros(Qn * self.c.ncell)
        lbm.lbm_populations(self.h, f, g, 0)
        fr, gr = o.populations()
        assert rel_linf(f, fr.ravel()) <= tol
        assert rel_linf(g, gr.ravel()) <= tol
        rho, u, T = np.zeros(self.c.ncell), np.zeros(self.c.dim * self.c.ncell), np.zeros(self.c.ncell)
        lbm.lbm_moments(self.h, rho, u, T, 0)
        rr, ur, Tr = o.moments()
        assert rel_linf(rho, rr) <= tol and rel_linf(T, Tr) <= tol
        tol_u = tol if f32 else tol * max(float(np.max(np.abs(ur))), 1e-3)
        assert float(np.max(np.abs(u - ur.ravel()))) <= tol_u

    def close(self):
        lbm.lbm_destroy(self.h)


def _oracle(c, F, Q):
    o = orc.Oracle(oracle_params(c))
    o.init(*c.fields())
    o.set_fields(F, Q)
    return o


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_fields_2d_match_oracle(storage, tol):
    c = wl.vdw_spinodal(n=37, ny=29, storage=storage)
    F, Q = _fields(c, 5)
    r = _Run(c, F, Q)
    assert lbm.lbm_get_kernel(r.h)[0] == lbm.LBM_KERNEL_SPLIT
    r.step(25)
    o = _oracle(c, F, Q)
    o.step(25)
    r.compare(o, tol, f32=storage == "f32")
    r.close()


def test_fields_3d_walls_match_oracle():
    c = wl.pr_heated_slab(n=9, nz=8, storage="f64")
    F, Q = _fields(c, 6)
    r = _Run(c, F, Q)
    assert lbm.lbm_get_kernel(r.h)[0] == lbm.LBM_KERNEL_SPLIT
    with pytest.raises(lbm.LbmError, match="split"):
        lbm.lbm_set_kernel(r.h, lbm.LBM_KERNEL_ZMARCH)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_kernel(r.h, lbm.LBM_KERNEL_FUSED)
    r.step(20)
    o = _oracle(c, F, Q)
    o.step(20)
    r.compare(o, 1e-12)
    r.close()


def test_field_changed_between_steps():
    # the kernels read the caller's field at every step: a new field takes effect from the next step
    import torch

    c = wl.acoustic_shear(n=24, storage="f64")
    F, Q = _fields(c, 7)
    F2, Q2 = _fields(c, 8)
    r = _Run(c, F, Q)
    r.step(10)
    r.F.copy_(torch.from_numpy(F2))
    r.Q.copy_(torch.from_numpy(Q2))
    r.step(10)
    o = _oracle(c, F, Q)
    o.step(10)
    o.set_fields(F2, Q2)
    o.step(10)
    r.compare(o, 1e-12)
    r.close()
