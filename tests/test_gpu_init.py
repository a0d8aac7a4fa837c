"""lbm_init through the C ABI: host inputs (pageable or pinned) and device
inputs give the same state bit for bit, and fields with rho <= 0, T <= 0 or a
NaN are rejected with LBM_E_INVALID from every input kind and storage type,
after which the handle steps only once it has been initialised again."""
import numpy as np
import pytest

from paper_2609_28679_b300 import lbm
from paper_2609_28679_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _inputs(case, kind):
    import torch

    rho, u, T = case.fields()
    arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (rho, u, T)]
    if kind == "pageable":
        return arrs, 0
    if kind == "pinned":
        pinned = [torch.from_numpy(a).pin_memory() for a in arrs]
        return pinned, 0
    return [torch.from_numpy(a).cuda() for a in arrs], 1


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_init_host_pinned_and_device_inputs_agree(storage):
    import torch

    # the split kernels sum in a fixed order (the fused scatter's shared-memory
    # atomics do not), so equal inputs give equal bits
    case = wl.vdw_spinodal(40, steps=3, storage=storage)
    ref = None
    for kind in ("pageable", "pinned", "device"):
        sim = lbm.Simulation(case, variant=lbm.LBM_KERNEL_SPLIT)
        (rho, u, T), on_dev = _inputs(case, kind)
        lbm.lbm_init(sim.h, rho, u, T, on_dev)
        torch.cuda.synchronize()
        sim.step(3)
        f, g = sim.populations()
        sim.close()
        if ref is None:
            ref = (f, g)
        else:
            assert np.array_equal(f, ref[0]) and np.array_equal(g, ref[1]), kind


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("kind", ["pageable", "pinned", "device"])
@pytest.mark.parametrize("bad", ["rho_zero", "T_negative", "rho_nan"])
def test_init_rejects_nonpositive_fields(storage, kind, bad):
    import torch

    case = wl.vdw_spinodal(24, steps=2, storage=storage)
    sim = lbm.Simulation(case, variant=lbm.LBM_KERNEL_FUSED)
    (rho, u, T), on_dev = _inputs(case, kind)
    k = case.ncell // 3 + 5  # one interior cell
    good_rho, good_T = rho.clone() if on_dev or kind == "pinned" else rho.copy(), None
    if bad == "rho_zero":
        rho[k] = 0.0
    elif bad == "rho_nan":
        rho[k] = float("nan")
    else:
        good_T = T.clone() if on_dev or kind == "pinned" else T.copy()
        T[k] = -1.0
    with pytest.raises(lbm.LbmError, match="must be > 0"):
        lbm.lbm_init(sim.h, rho, u, T, on_dev)
    with pytest.raises(lbm.LbmError):
        sim.step(1)  # the handle is not initialised after a rejected init
    if good_T is not None:
        T = good_T
    lbm.lbm_init(sim.h, good_rho, u, T, on_dev)
    torch.cuda.synchronize()
    sim.step(2)
    assert int(sim.diagnostics()[0]) == 0
    r, _, _ = sim.moments()
    assert np.all(np.isfinite(r)) and np.all(r > 0)
    sim.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("kind", ["pageable", "pinned", "device"])
def test_float32_io_matches_float64_io(storage, kind):
    # lbm_init_f32 / lbm_moments_f32: from float32 fields the state is bit-equal to
    # lbm_init from the same values in float64 (the state is formed in float32 either
    # way, and the 16-bit offsets come from the same float64 means), and the exported
    # float32 moments are exactly the float64 export rounded (it holds float32 values)
    import torch

    case = wl.vdw_spinodal(40, steps=3, storage=storage)
    (rho, u, T), on_dev = _inputs(case, kind)
    as32 = [torch.as_tensor(a).to(torch.float32) for a in (rho, u, T)]
    as64 = [a.to(torch.float64) for a in as32]
    if kind == "pageable":
        as32 = [a.numpy() for a in as32]
        as64 = [a.numpy() for a in as64]
    elif kind == "pinned":
        as32 = [a.cpu().pin_memory() for a in as32]
        as64 = [a.cpu().pin_memory() for a in as64]
    out = []
    for single in (False, True):
        sim = lbm.Simulation(case, variant=lbm.LBM_KERNEL_SPLIT)
        if single:
            lbm.lbm_init_f32(sim.h, *as32, on_dev)
        else:
            lbm.lbm_init(sim.h, *as64, on_dev)
        sim.step(3)
        f, g = sim.populations()
        r64, u64, T64 = sim.moments()
        n = case.ncell
        r32, u32, T32 = np.zeros(n, np.float32), np.zeros(2 * n, np.float32), np.zeros(n, np.float32)
        lbm.lbm_moments_f32(sim.h, r32, u32, T32, 0)
        sim.close()
        out.append((f, g, r64, u64, T64, r32, u32, T32))
    (f0, g0, r64, u64, T64, _, _, _), (f1, g1, _, _, _, r32, u32, T32) = out
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    assert np.array_equal(r32, r64.astype(np.float32))
    assert np.array_equal(u32, u64.astype(np.float32))
    assert np.array_equal(T32, T64.astype(np.float32))


def test_float32_io_rejects_float64_arrays_and_bad_fields():
    case = wl.vdw_spinodal(24, steps=2, storage="f32")
    sim = lbm.Simulation(case, variant=lbm.LBM_KERNEL_FUSED)
    rho, u, T = case.fields()
    with pytest.raises(lbm.LbmError, match="float32"):
        lbm.lbm_init_f32(sim.h, rho, u.ravel(), T, 0)
    r32 = np.ascontiguousarray(rho, dtype=np.float32)
    u32 = np.ascontiguousarray(u.ravel(), dtype=np.float32)
    T32 = np.ascontiguousarray(T, dtype=np.float32)
    r32[7] = 0.0
    with pytest.raises(lbm.LbmError, match="must be > 0"):
        lbm.lbm_init_f32(sim.h, r32, u32, T32, 0)
    sim.close()


def test_host_transfers_in_parts_match_device_transfers_3d():
    # 160^3 (4.1 M cells): lbm_init_f32 from pinned host memory and lbm_moments_f32 to it
    # go in three parts (copies beside k_init, and beside the gathering z-march's first
    # pass and the export); the state and the moments equal those from and to the device
    import torch

    case = wl.pr_droplet(160, storage="f32", radius=20.0)
    rho, u, T = case.fields()
    host = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).pin_memory() for a in (rho, u, T)]
    dev = [a.cuda() for a in host]
    n = case.ncell
    out = []
    for on_dev in (0, 1):
        sim = lbm.Simulation(case)
        assert sim.kernel()[0] == lbm.LBM_KERNEL_ZGATHER
        lbm.lbm_init_f32(sim.h, *(dev if on_dev else host), on_dev)
        sim.step(2)
        if on_dev:
            res = [torch.zeros(m, dtype=torch.float32, device="cuda") for m in (n, 3 * n, n)]
            lbm.lbm_moments_f32(sim.h, *res, 1)
            res = [r.cpu().numpy() for r in res]
        else:
            res = [torch.zeros(m, dtype=torch.float32).pin_memory() for m in (n, 3 * n, n)]
            lbm.lbm_moments_f32(sim.h, *res, 0)
            res = [r.numpy().copy() for r in res]
        sim.close()
        out.append(res)
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert np.all(out[0][0] > 0) and np.all(out[0][2] > 0)


@pytest.mark.parametrize("variant", [lbm.LBM_KERNEL_SPLIT, lbm.LBM_KERNEL_YMARCH])
def test_host_transfers_in_parts_match_device_transfers_batch(variant):
    # a 2-D batch of uneven simulations, 2.3 M cells: two parts, the boundary inside
    # the first simulation; float64 pageable host fields against device fields (kernels
    # that sum in a fixed order, so equal inputs give equal bits; the row march carries
    # moments, which the host upload prepares run by run and the device one at the first step)
    import torch

    cases = [wl.vdw_spinodal(n=1500, ny=900, storage="f32", seed=11), wl.vdw_spinodal(n=700, ny=500, storage="f32", seed=12),
             wl.vdw_spinodal(n=1000, ny=600, storage="f32", seed=13)]
    fs = [c.fields() for c in cases]
    rho = np.concatenate([f[0] for f in fs]).astype(np.float64)
    u = np.concatenate([f[1].ravel() for f in fs]).astype(np.float64)
    T = np.concatenate([f[2] for f in fs]).astype(np.float64)
    out = []
    for on_dev in (0, 1):
        sim = lbm.Simulation(cases, variant=variant)
        if on_dev:
            lbm.lbm_init(sim.h, *[torch.from_numpy(a).cuda() for a in (rho, u, T)], 1)
        else:
            lbm.lbm_init(sim.h, rho, u, T, 0)
        sim.step(2)
        f, g = sim.populations()
        if on_dev:
            res = [torch.zeros(m, dtype=torch.float64, device="cuda") for m in (rho.size, u.size, T.size)]
            lbm.lbm_moments(sim.h, *res, 1)
            res = [r.cpu().numpy() for r in res]
        else:
            res = list(sim.moments())
        sim.close()
        out.append((f, g, res))
    (f0, g0, m0), (f1, g1, m1) = out
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    for a, b in zip(m0, m1):
        assert np.array_equal(a, b)
