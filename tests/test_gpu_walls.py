"""Non-equilibrium-extrapolation walls (zwalls = 2, the wall treatment of the
thermal Couette flow, App. B) on the GPU split kernels, through the C ABI,
against the FP64 CPU oracle on the same seeded inputs: populations and
moments element by element, the conservation totals, a batch of uneven
simulations, the steady Couette profile, and the API rules (walls set before
stepping, split kernels only).

Tolerances as in the other parity tests: float64 1e-12 relative (u to 1e-12 of
max(max|u_ref|, 1e-3)), float32 1e-5 (u to 1e-5 of the lattice speed),
16-bit storage by its stored precision."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_28679_b300 import lbm
from paper_2609_28679_b300 import workloads as wl
from tests.util import oracle_params, rel_linf

pytestmark = pytest.mark.gpu


def _wall_case(eos="vdw", nx=5, ny=4, nz=12, storage="f64", wall_rho=0, phi_central=0, **kw):
    base = dict(name="nee", dim=3, nx=nx, ny=ny, nz=nz, zwalls=2, R=1.0, cv=2.5, k_over_mu=3.5,
                eta_over_mu=0.5, accel=(2e-5, 0.0, -1e-5), phi_central=phi_central,
                uw_lo=(0.0, 0.01, 0.0), uw_hi=(0.03, 0.0, 0.0), wall_rho=wall_rho, storage=storage)
    if eos == "vdw":
        base.update(eos="vdw", a=wl.VDW_A, b=wl.VDW_B, kappa=wl.VDW_KAPPA, Tw_lo=0.1, Tw_hi=0.104,
                    init=dict(kind="couette", rho0=1.2, amp=0.02, seed=21))
    elif eos == "pr":
        # supercritical (T/Tc = 1.1): a wall colder than the saturation temperature would condense vapour
        base.update(eos="pr", Tc=wl.PR_TC, Pc=wl.PR_PC, omega=wl.PR_OMEGA, kappa=0.01, Tw_lo=0.55,
                    Tw_hi=0.57, q=2e-6, zlo=0, zhi=3, init=dict(kind="couette", rho0=0.4, amp=0.02, seed=22))
    else:
        base.update(eos="ideal", Tw_lo=0.33, Tw_hi=0.35, init=dict(kind="couette", rho0=3.0, amp=0.02, seed=23))
    base.update(kw)
    return wl.Case(**base)


SPLIT, ZMARCH = lbm.LBM_KERNEL_SPLIT, lbm.LBM_KERNEL_ZMARCH
# split kernels, and the z-march with the default range and with 4-plane ranges (several per column)
VARIANTS = [SPLIT, (ZMARCH, (30, 14, 32)), (ZMARCH, (30, 6, 4))]


def _pair(c, steps, fields=None, variant=SPLIT):
    fields = fields if fields is not None else c.fields()
    sim = lbm.Simulation(c)
    tile = (0, 0, 0)
    if isinstance(variant, tuple):
        variant, tile = variant
    lbm.lbm_set_kernel(sim.h, variant, *tile)
    assert sim.kernel()[0] == variant
    sim.init(fields)
    sim.step(steps)
    o = orc.Oracle(oracle_params(c))
    o.init(*fields)
    o.step(steps)
    return sim, o


def _compare(sim, o, tol, f32=False):
    f, g = sim.populations()
    fr, gr = o.populations()
    assert rel_linf(f, fr.ravel()) <= tol
    assert rel_linf(g, gr.ravel()) <= tol
    rho, u, T = sim.moments()
    rr, ur, Tr = o.moments()
    assert rel_linf(rho, rr) <= tol
    assert rel_linf(T, Tr) <= tol
    tol_u = tol if f32 else tol * max(float(np.max(np.abs(ur))), 1e-3)
    assert float(np.max(np.abs(u - ur.ravel()))) <= tol_u


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("wall_rho", [0, 1, 2])
@pytest.mark.parametrize("eos", ["ideal", "vdw", "pr"])
def test_f64_walls_match_oracle(eos, wall_rho, variant):
    c = _wall_case(eos, wall_rho=wall_rho)
    sim, o = _pair(c, 25, variant=variant)
    _compare(sim, o, 1e-12)


@pytest.mark.parametrize("variant", VARIANTS)
def test_f64_walls_central_phi_ragged_plane(variant):
    # 7 x 3 planes (one block holds cells of several z layers), central Phi
    c = _wall_case("vdw", nx=7, ny=3, nz=9, phi_central=1)
    sim, o = _pair(c, 30, variant=variant)
    _compare(sim, o, 1e-12)


def test_f64_walls_invariants_match_oracle():
    c = _wall_case("pr")
    sim, o = _pair(c, 15)
    gi = sim.invariants()[0]
    oi = o.invariants()
    assert np.all(np.abs(gi - oi) <= 1e-12 * np.maximum(np.abs(oi), np.abs(oi[0])))


def test_f64_walls_batch_of_uneven_simulations():
    cases = [_wall_case("vdw", nx=n, ny=n + 1, nz=n + 4, init=dict(kind="couette", rho0=1.2, amp=0.02, seed=n))
             for n in (3, 6, 4)]
    sim = lbm.Simulation(cases)
    sim.init()
    sim.step(12)
    rho, u, T = sim.moments()
    off = 0
    for c in cases:
        o = orc.Oracle(oracle_params(c))
        o.init(*c.fields())
        o.step(12)
        rr, ur, Tr = o.moments()
        n = c.ncell
        assert rel_linf(rho[off:off + n], rr) <= 1e-12
        assert rel_linf(T[off:off + n], Tr) <= 1e-12
        assert np.max(np.abs(u[3 * off:3 * off + 3 * n] - ur.ravel())) <= 1e-13
        off += n


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("eos", ["ideal", "vdw"])
def test_f32_walls_match_oracle(eos, variant):
    c = _wall_case(eos, storage="f32", phi_central=1)
    sim, o = _pair(c, 25, variant=variant)
    _compare(sim, o, 1e-5, f32=True)


def test_default_kernels_for_walls():
    # 32- and 64-bit storage: the z-march; 16-bit storage: the split kernels
    for storage, want in (("f64", ZMARCH), ("f32", ZMARCH), ("bf16", SPLIT)):
        sim = lbm.Simulation(_wall_case("ideal", storage=storage))
        assert sim.kernel()[0] == want, storage
        sim.close()


def test_bf16_walls_error_bound():
    # 16-bit storage keeps f - f^ref: the stored deviation has 2^-9 relative precision per step
    c = _wall_case("ideal", storage="bf16", phi_central=1)
    sim, o = _pair(c, 10)
    f, g = sim.populations()
    fr, gr = o.populations()
    assert rel_linf(f, fr.ravel()) <= 2e-3
    assert rel_linf(g, gr.ravel()) <= 2e-3


@pytest.mark.parametrize("storage,tol", [("f64", 0.01), ("f32", 0.02)])
def test_thermal_couette_steady_profile(storage, tol):
    # the paper's analytic profile (App. B): T = T_C + (T_H - T_C) xi + U^2 / (2 k/mu) xi (1 - xi)
    nz, U, kmu = 17, 0.2, 1.75
    c = wl.Case(name="couette", dim=3, nx=2, ny=2, nz=nz, zwalls=2, eos="ideal", R=1.0, cv=2.5, k_over_mu=kmu,
                 phi_central=1, uw_hi=(U, 0.0, 0.0), Tw_lo=0.33, Tw_hi=0.35, storage=storage,
                 init=dict(kind="couette", rho0=3.0))
    sim = lbm.Simulation(c)
    sim.init()
    sim.step(4000)
    rho, u, T = sim.moments()
    xi = (np.arange(c.ncell) // (c.nx * c.ny)) / (nz - 1)
    ana = 0.33 + 0.02 * xi + U * U / (2 * kmu) * xi * (1 - xi)
    bump = U * U / (8 * kmu)
    assert np.max(np.abs(T - ana)) <= tol * bump
    assert np.max(np.abs(u.reshape(3, -1)[0] - U * xi)) <= (1e-10 if storage == "f64" else 1e-4) * U


def test_walls_must_be_set_and_run_split_only():
    c = _wall_case("ideal")
    lat, eos, force, heat = lbm.structs_from_case(c)
    h = lbm.lbm_create(lat, eos, c.tau_f, c.tau_g, force, heat)
    try:
        rho, u, T = c.fields()
        lbm.lbm_init(h, rho, u.ravel(), T, 0)
        with pytest.raises(lbm.LbmError, match="lbm_set_walls"):
            lbm.lbm_step(h, 1)
        with pytest.raises(lbm.LbmError, match="split"):
            lbm.lbm_set_kernel(h, lbm.LBM_KERNEL_FUSED)
        with pytest.raises(lbm.LbmError, match="30x14"):
            lbm.lbm_set_kernel(h, lbm.LBM_KERNEL_ZMARCH, 62, 14, 32)
        lbm.lbm_set_kernel(h, lbm.LBM_KERNEL_AUTO)
        assert lbm.lbm_get_kernel(h)[0] == lbm.LBM_KERNEL_SPLIT
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_walls(h, (0, 0, 0), -1.0, (0, 0, 0), 0.3)
        lbm.lbm_set_walls(h, c.uw_lo, c.Tw_lo, c.uw_hi, c.Tw_hi)
        lbm.lbm_step(h, 2)
    finally:
        lbm.lbm_destroy(h)
    # a handle without such walls refuses a wall state
    p = wl.pr_heated_slab(n=8, nz=6, storage="f64")
    sim = lbm.Simulation(p)
    with pytest.raises(lbm.LbmError, match="no simulation"):
        lbm.lbm_set_walls(sim.h, (0, 0, 0), 0.3, (0, 0, 0), 0.3)
    sim.close()


def test_autotune_with_walls_restores_the_state():
    # the trial steps rewrite the boundary slots of the current populations; the snapshot restores them
    c = _wall_case("vdw", nx=40, ny=20, nz=24, storage="f32", phi_central=1)
    sim = lbm.Simulation(c)
    sim.init()
    sim.step(3)
    f0, g0 = sim.populations()
    (variant, tx, ty, tz), ms = sim.autotune(3)
    assert variant in (SPLIT, ZMARCH) and ms > 0
    if variant == ZMARCH:
        assert (tx, ty) in ((30, 14), (30, 6))
    f1, g1 = sim.populations()
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    sim.step(4)
    o = orc.Oracle(oracle_params(c))
    o.init(*c.fields())
    o.step(7)
    assert rel_linf(sim.moments()[0], o.moments()[0]) <= 1e-5
