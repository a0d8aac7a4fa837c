"""Benchmark of the fused DDF lattice Boltzmann step on B300.

Workload (one "step" = one time step of the whole hot path): the 2-D van der
Waals liquid-vapour quench on a 512 x 512 D2Q9 lattice with float32
populations, Korteweg capillarity, gravity and the explicit temperature
inversion (the paper-shaped configuration the MLUPS metric is quoted on).
Inputs are synthetic and seeded (paper_2609_28679_b300.workloads).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (no data-path collective); value = cells x steps of
all ranks / max over ranks of the timed region.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (million lattice-cell updates per second, f and g populations)"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6400.0
NOMINAL_HBM_GBS = 8000.0  # B300 HBM3e, nominal (context for the measured fraction)
L2_FLUSH_BYTES = 256 << 20


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.4 TB/s, no MEASURED_PEAKS.json)"


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("lbm_device.cuh", "lbm_fused.cuh"):
        with open(os.path.join(ROOT, "paper_2609_28679_b300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str, workload: str):
    """DRAM bytes and ncu duration (us) per launch from the committed ncu
    summary, if it was taken on the current kernel source (else None, None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None, None
    src = _kernel_source_hash()
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload \
                    and parts[2] == src:
                return float(parts[3]), (float(parts[4]) if len(parts) >= 5 else None)
    return None, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms (the timed
    region lasts long enough for several samples at the default step count)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi needs a moment before its first sample: wait for it, so
        # that the samples cover the timed region from its start
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 10.0 and self.proc.poll() is None:
            if os.path.getsize(self.file.name) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_mlups(case, steps_budget_s: float, threads: int | None = None):
    """Time the FP64 CPU oracle on the workload (bounded number of full steps)."""
    from oracle import oracle as orc

    if threads:
        orc.set_threads(threads)
    o = orc.Oracle(orc.params_from_case(case))
    o.init(*case.fields())
    t0 = time.perf_counter()
    o.step(1)  # warm-up step (also sizes the sample)
    t1 = time.perf_counter() - t0
    n = max(1, min(200, int(steps_budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return case.ncell * n / dt / 1e6, n, dt, orc.get_threads()


def _oracle_threads(n: int) -> None:
    from oracle import oracle as orc

    orc.set_threads(n)


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def max_over_ranks(x: float) -> float:
    """Maximum of x over the ranks of the default process group (x itself
    without one): the timed region of a weak-scaling replica run is the
    slowest rank's."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(cells_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job MLUPS of `world` replicas timed over max_ms."""
    return world * cells_per_rank * steps / (max_ms * 1e-3) / 1e6


def _time_steps(torch, sim, steps, stream=None, per_step=True):
    """ms per step over `steps` steps (device events).  per_step: one event
    pair per step with L2 flushed before each (workloads that fit in L2);
    else one pair around all steps, L2 flushed once (inputs larger than L2,
    or steps replayed as CUDA graphs)."""
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    st = stream or torch.cuda.current_stream()
    if per_step:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(st)
            sim.step(1)
            b.record(st)
        torch.cuda.synchronize()
        del flush
        return sum(a.elapsed_time(b) for a, b in ev) / steps
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    sim.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    del flush
    return e0.elapsed_time(e1) / steps


def _form(lbm, torch, case, steps, storage_bytes, graphs=0, mlp=None, tune=True, warm=3, pops=2):
    """MLUPS, ms per step and HBM fraction of one workload form (pops: population
    sets read and written per step, 2 for f and g, 1 in the isothermal mode)."""
    sim = lbm.Simulation(case)
    stream = None
    if graphs:
        stream = torch.cuda.Stream()
        sim.use_graphs(graphs, stream)
    if mlp is not None:
        lbm.lbm_mlp_load(sim.h, mlp)
    ctx = torch.cuda.stream(stream) if stream is not None else _null()
    with ctx:
        sim.init()
        if tune:
            sim.autotune(3)
        sim.step(warm)
        # population bytes of one step; below the 126 MB L2 every timed step starts cold
        Q = 3 ** sim.dim
        pop_bytes = 2 * pops * Q * storage_bytes * sum(c.ncell for c in sim.cases)
        ms = _time_steps(torch, sim, steps, stream, per_step=(not graphs and pop_bytes < 4 * L2_FLUSH_BYTES))
        rho, u, T = sim.moments()
        diag = sim.diagnostics()
    n = sum(c.ncell for c in sim.cases)
    Q = 3 ** sim.dim
    alg = 2 * pops * Q * storage_bytes * n
    peak, _ = _peaks()
    out = {"cells": n, "ms_per_step": ms, "mlups": n / (ms * 1e3), "hbm_frac": alg / (ms * 1e-3) / 1e9 / peak,
           "kernel": list(sim.kernel()), "steps_timed": steps, "diagnostics": [int(v) for v in diag]}
    sim.close()
    return out, (rho, T)


class _null:
    def __enter__(self):
        return None

    def __exit__(self, *a):
        return False


def _rel_dev(a, b) -> float:
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _vs_f64(ref, ref_fields, r, fields):
    """Speed-up over the float64 GPU run of the same workload, and the
    deviation from it after the same steps from the same state."""
    r["speedup_vs_f64_gpu"] = ref["ms_per_step"] / r["ms_per_step"]
    r["rel_dev_vs_f64_gpu"] = {"rho": _rel_dev(fields[0], ref_fields[0]), "T": _rel_dev(fields[1], ref_fields[1])}


def _measure_forms(lbm, wl, torch, steps):
    """Every form on its full-size workload (few steps each), next to the
    plain float64 GPU path of the same workload: MLUPS, HBM fraction, speed-up
    and deviation from float64 after the same steps."""
    res = {}
    try:
        r, _ = _form(lbm, torch, wl.acoustic_shear(128, storage="f64"), steps, 8)
        res["f64_ideal_2d_128"] = r
        # the 512^2 van der Waals quench (the bench workload)
        r64, f64 = _form(lbm, torch, wl.vdw_spinodal(512, storage="f64"), steps, 8, warm=0)
        res["f64_vdw_512"] = r64
        r, fr = _form(lbm, torch, wl.vdw_spinodal(512, storage="f32"), steps, 4, warm=0)
        _vs_f64(r64, f64, r, fr)
        res["f32_vdw_512"] = r
        # the isothermal mode (f only; algorithmic bytes 2 Q s) beside the full model
        iso = wl.vdw_spinodal(512, storage="f32")
        iso.isothermal = 1
        ri, _ = _form(lbm, torch, iso, steps, 4, warm=0, pops=1)
        ri["speedup_vs_full_model"] = r["ms_per_step"] / ri["ms_per_step"]
        res["f32_vdw_512_isothermal"] = ri
        # 64 simulations per launch under CUDA graphs
        b64, fb64 = _form(lbm, torch, wl.vdw_batch(64, storage="f64"), steps, 8, graphs=10, warm=0)
        res["f64_vdw_batch_64"] = b64
        r, fr = _form(lbm, torch, wl.vdw_batch(64, storage="f32"), steps, 4, graphs=10, warm=0)
        _vs_f64(b64, fb64, r, fr)
        res["f32_vdw_batch_64"] = r
        torch.cuda.empty_cache()
        # 3-D heated slab: float64, float32, and 16-bit storage with offsets
        s64, fs64 = _form(lbm, torch, wl.pr_heated_slab(256, storage="f64"), steps, 8, warm=0)
        res["f64_pr_slab_256"] = s64
        for st, sb in (("f32", 4), ("bf16", 2), ("f16", 2)):
            r, fr = _form(lbm, torch, wl.pr_heated_slab(256, storage=st), steps, sb, warm=0)
            _vs_f64(s64, fs64, r, fr)
            res[f"{st}_pr_slab_256"] = r
        # the paper's tau = mu / P per cell (beta per cell): mu = 0.8 P of the initial vapour state
        cmu = wl.pr_heated_slab(256, storage="f32")
        cmu.mu = 0.8 * 0.0942393
        rm, _ = _form(lbm, torch, cmu, steps, 4, warm=0)
        rm["speedup_vs_constant_tau"] = res["f32_pr_slab_256"]["ms_per_step"] / rm["ms_per_step"]
        res["f32_pr_slab_256_constant_mu"] = rm
        iso = wl.pr_heated_slab(256, storage="f32")
        iso.isothermal, iso.q = 1, 0.0
        ri, _ = _form(lbm, torch, iso, steps, 4, warm=0, pops=1)
        ri["speedup_vs_full_model"] = res["f32_pr_slab_256"]["ms_per_step"] / ri["ms_per_step"]
        res["f32_pr_slab_256_isothermal"] = ri
        del fs64
        torch.cuda.empty_cache()
        # extrapolation walls (z-march) and a friction duct (split kernels): thermal Couette, Fanno duct
        res["f32_thermal_couette_256x256x128"], _ = _form(lbm, torch, wl.thermal_couette(256, 128),
                                                               steps, 4, tune=False, warm=2)
        res["f32_fanno_duct_128x128x256"], _ = _form(lbm, torch, wl.fanno_duct(128, 256), steps, 4,
                                                          tune=False, warm=2)
        torch.cuda.empty_cache()
        # 3-D droplet: Newton in float64 and float32, and the learned temperature start
        nd = max(4, steps // 2)
        d64, fd64 = _form(lbm, torch, wl.pr_droplet(384, storage="f64"), nd, 8, warm=0)
        res["f64_pr_droplet_384_newton"] = d64
        torch.cuda.empty_cache()
        drop = wl.pr_droplet(384, storage="f32")
        newton, fdn = _form(lbm, torch, drop, nd, 4, warm=0)
        _vs_f64(d64, fd64, newton, fdn)
        res["f32_pr_droplet_384_newton"] = newton
        le = lbm.structs_from_case(drop)[1]
        params = np.zeros(lbm.lbm_mlp_nparams(), dtype=np.float32)
        t0 = time.perf_counter()
        lbm.lbm_mlp_train(le, (0.1, 2.6, 0.85, 1.05), 1_000_000, 2000, 1024, 2e-3, 7, True, params)
        train_s = time.perf_counter() - t0
        drop_m = wl.pr_droplet(384, storage="f32")
        drop_m.t_solver = 1
        r, fr = _form(lbm, torch, drop_m, nd, 4, mlp=params, warm=0)
        _vs_f64(d64, fd64, r, fr)
        r["train_s"] = train_s
        r["speedup_vs_f32_newton"] = newton["ms_per_step"] / r["ms_per_step"]
        r["rel_dev_vs_f32_newton"] = {"rho": _rel_dev(fr[0], fdn[0]), "T": _rel_dev(fr[1], fdn[1])}
        res["f32_pr_droplet_384_mlp"] = r
        torch.cuda.empty_cache()
    except Exception as e:  # report what was measured
        res["error"] = f"{type(e).__name__}: {e}"
    return res


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_2609_28679_b300 import workloads as wl

    case = wl.vdw_spinodal(512, storage="f64")
    budget = min(120.0, 2.0 * max(args.steps, 1))
    value, n, dt, cores = _oracle_mlups(case, budget)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / n * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "vdw_spinodal_512: 2-D van der Waals quench, 512x512 D2Q9, Korteweg + gravity",
                   "cells": case.ncell},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} full time steps of the 512x512 workload (FP64 C oracle, OpenMP)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2609_28679_b300 import lbm
    from paper_2609_28679_b300 import workloads as wl

    rank, world, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    case = wl.vdw_spinodal(512, storage="f32")
    sim = lbm.Simulation(case)
    sim.init()
    if args.kernel == "auto":
        # warm-up includes the autotuner (kernel variant and tile for this workload; state restored)
        sim.autotune(5)
    else:
        kind, _, tile = args.kernel.partition(":")
        t = [int(v) for v in tile.split("x")] if tile else [0, 0, 0]
        lbm.lbm_set_kernel(sim.h, lbm.LBM_KERNEL_FUSED if kind == "fused" else lbm.LBM_KERNEL_SPLIT,
                           *(t + [0] * (3 - len(t))))
    variant, tx, ty, tz = sim.kernel()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        sim.step(1)
    torch.cuda.synchronize()

    # device-timed region: one event pair per step, L2 flushed between steps (outside the pairs)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        sim.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms)
    diag = sim.diagnostics()

    # end to end through the C ABI with host buffers: upload the state, one step, read the fields back
    rho, u, T = case.fields()
    rho_h = torch.from_numpy(rho).pin_memory().numpy()
    u_h = torch.from_numpy(np.ascontiguousarray(u.ravel())).pin_memory().numpy()
    T_h = torch.from_numpy(T).pin_memory().numpy()
    out_r = torch.empty(case.ncell, dtype=torch.float64).pin_memory().numpy()
    out_u = torch.empty(2 * case.ncell, dtype=torch.float64).pin_memory().numpy()
    out_T = torch.empty(case.ncell, dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(3, min(args.steps, 50))
    for it in range(2):
        lbm.lbm_init(sim.h, rho_h, u_h, T_h, 0)
        lbm.lbm_step(sim.h, 1)
        lbm.lbm_moments(sim.h, out_r, out_u, out_T, 0)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(e2e_steps):
        lbm.lbm_init(sim.h, rho_h, u_h, T_h, 0)
        lbm.lbm_step(sim.h, 1)
        lbm.lbm_moments(sim.h, out_r, out_u, out_T, 0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    sim.close()

    forms = None
    if not args.no_forms:
        forms = _measure_forms(lbm, wl, torch, min(args.steps, 20))

    Q = 9
    alg_bytes = 4 * Q * 4 * case.ncell  # read + write f and g once, float32
    avg_ms = total_ms / args.steps
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    peak, peak_src = _peaks()
    kname = "k_fused" if variant == lbm.LBM_KERNEL_FUSED else "k_collide"
    value = aggregate_mlups(case.ncell, args.steps, world, total_ms)
    traffic, ncu_us = _ncu_traffic(kname, "vdw_spinodal_512_f32")
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cb_case = wl.vdw_spinodal(512, storage="f64")
            cv, n, dt, cores = _oracle_mlups(cb_case, 15.0)
            cv1, n1, dt1, _ = _oracle_mlups(cb_case, 8.0, threads=1)
            _oracle_threads(cores)
            cpu = {"value": cv, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{n} full time steps of the same 512x512 workload ({dt:.1f} s, FP64 C oracle, OpenMP)",
                   "single_core": {"value": cv1, "unit": UNIT, "sample": f"{n1} full time steps ({dt1:.1f} s)"},
                   "cpu_model": _cpu_model(), "nproc": os.cpu_count()}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; paper-shaped vdW quench)",
            "config": {"workload": "vdw_spinodal_512: 2-D van der Waals quench, 512x512 D2Q9, f32 populations, "
                                   "Korteweg capillarity + gravity", "cells": case.ncell, "storage": "f32",
                       "kernel": kname, "tile": [tx, ty, tz],
                       "l2": "flushed between timed steps (256 MiB write outside the event pairs)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src,
                         "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                         "ncu_dram_gbs": (traffic / (ncu_us * 1e-6) / 1e9) if traffic and ncu_us else None,
                         "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": avg_ms},
            "e2e": {"value": case.ncell * e2e_steps / e2e_s / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": int(rho_h.nbytes + u_h.nbytes + T_h.nbytes),
                    "d2h_bytes_per_step": int(out_r.nbytes + out_u.nbytes + out_T.nbytes),
                    "what": "lbm_init from pinned host fields + lbm_step(1) + lbm_moments to pinned host, per step"},
            "gpu_launches": args.steps * (1 if variant == lbm.LBM_KERNEL_FUSED else 3),
            "clocks": clk,
            "cpu_baseline": cpu,
            "diagnostics": {"nonfinite": int(diag[0]), "theta_le_0": int(diag[1]), "newton_cap": int(diag[2])},
            "forms": forms,
            "wall_s_timed_region": t_wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the per-form measurements")
    ap.add_argument("--kernel", default="auto",
                    help="auto (autotuned), split, or fused:TXxTY[xTZ] (pinned, e.g. for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
