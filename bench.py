"""Benchmark of the DDF lattice Boltzmann step on B300.

Workload (one "step" = one time step of the whole hot path): the largest
configuration, the 3-D Peng-Robinson droplet on a 384^3 D3Q27 lattice
(56.6 M cells, density ratio 8, Korteweg capillarity, heat source) with
float32 populations and collision arithmetic and the Newton temperature
inversion warm-started from the previous step.  The other forms (float64,
16-bit storage, the learned temperature start, the batched 2-D form, the
512^2 2-D quench ...) are measured after it and reported under "forms".
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
HEADLINE = "pr_droplet_384"
# the workload's constants in lattice units (rescaled for stability, see workloads.py)
HEADLINE_DESC = ("pr_droplet_384: 3-D Peng-Robinson droplet, 384^3 D3Q27 periodic, float32 populations and collision, "
                 "Newton T(rho, e) warm-started; radius 48, rho_l/rho_v = 2.10988/0.26314, T/Tc = 0.9, omega 0.1; "
                 "temperature scale 1/20 of the slab's (Tc = 0.025, Pc = 0.00768503, kappa = 0.01, Q = 2.5e-8), "
                 "eta/mu = 10, k/mu = 3.5, tau = 0.8, central Phi")


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


# sources of each timed kernel: the ncu traffic figure counts only while they and the
# compile flags (build.py) are unchanged
_KERNEL_SOURCES = {
    "k_zgather": ("lbm_device.cuh", "lbm_async.cuh", "lbm_zgather.cuh"),
    "k_zmacro": ("lbm_device.cuh", "lbm_split.cuh", "lbm_zmarch.cuh"),
    "k_fused": ("lbm_device.cuh", "lbm_fused.cuh"),
    "k_ymarch": ("lbm_device.cuh", "lbm_async.cuh", "lbm_ymarch.cuh"),
}


def _kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for name in _KERNEL_SOURCES.get(kernel, ("lbm_device.cuh",)) + ("../build.py",):
        with open(os.path.join(ROOT, "paper_2609_28679_b300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str, workload: str):
    """DRAM bytes and ncu duration (us) per launch from the committed ncu
    summary, if it was taken on the current kernel source (else None, None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None, None
    src = _kernel_source_hash(kernel)
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload \
                    and parts[2] == src:
                return float(parts[3]), (float(parts[4]) if len(parts) >= 5 else None)
    return None, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms (the timed
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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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


def _oracle_window(case, half: int):
    """The oracle on a bounded sample of a 3-D workload: the periodic window
    of 2*half cells per side centred on the droplet's interface (liquid,
    interface and vapour cells)."""
    from paper_2609_28679_b300 import workloads as wl

    cx = case.nx // 2 + int(round(case.init.get("radius", 0.0)))
    sub, fields, _ = wl.window(case, (cx, case.ny // 2, case.nz // 2), half)
    return sub, fields


def _oracle_mlups(case, steps_budget_s: float, threads: int | None = None, half: int = 48):
    """Time the FP64 CPU oracle on a bounded sample of the workload (whole
    time steps of a window of it for a 3-D case); returns MLUPS, steps,
    seconds, threads, and the sample's description."""
    from oracle import oracle as orc

    if threads:
        orc.set_threads(threads)
    sample = case
    fields = None
    what = f"full {case.nx}x{case.ny}" + (f"x{case.nz}" if case.dim == 3 else "") + " lattice"
    if case.dim == 3 and case.ncell > (2 * half) ** 3:
        sample, fields = _oracle_window(case, half)
        what = (f"{2 * half}^3 periodic window of the {case.nx}^3 workload centred on the droplet interface "
                f"({sample.ncell} cells)")
    o = orc.Oracle(orc.params_from_case(sample))
    o.init(*(fields if fields is not None else sample.fields()))
    t0 = time.perf_counter()
    o.step(1)  # warm-up step (also sizes the sample)
    t1 = time.perf_counter() - t0
    n = max(1, min(200, int(steps_budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return sample.ncell * n / dt / 1e6, n, dt, orc.get_threads(), what


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


def _pass_times(lbm, sim, steps):
    """Mean device ms per step of the step's passes (lbm_step_timed: events
    between the passes on the handle's stream) and of the whole step."""
    ms = lbm.lbm_step_timed(sim.h, steps)
    return {"pass1_ms": float(ms[0]), "pass2_ms": float(ms[1]), "pass3_ms": float(ms[2]), "step_ms": float(ms[3])}


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


def _form(lbm, torch, case, steps, storage_bytes, graphs=0, mlp=None, tune=True, warm=3, pops=2, passes=False):
    """MLUPS, ms per step and HBM fraction of one workload form (pops: population
    sets read and written per step, 2 for f and g, 1 in the isothermal mode).
    passes: also the per-pass device times (lbm_step_timed) and the achieved
    bandwidth of the collide-stream pass."""
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
        npass = max(2, steps // 2) if passes else 0
        pt = _pass_times(lbm, sim, npass) if passes else None
        rho, u, T = sim.moments()
        diag = sim.diagnostics()
    n = sum(c.ncell for c in sim.cases)
    Q = 3 ** sim.dim
    alg = 2 * pops * Q * storage_bytes * n
    peak, _ = _peaks()
    out = {"cells": n, "ms_per_step": ms, "mlups": n / (ms * 1e3), "hbm_frac": alg / (ms * 1e-3) / 1e9 / peak,
           "kernel": list(sim.kernel()), "steps_timed": steps, "diagnostics": [int(v) for v in diag],
           "steps_since_init": warm + steps + npass}  # the autotuner restores state and counters
    if pt:
        out["passes"] = pt
        out["collide_pass_gbs"] = alg / (pt["pass3_ms"] * 1e-3) / 1e9
        out["collide_pass_hbm_frac"] = out["collide_pass_gbs"] / peak
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


def _fp64_bound(r, fp64_peak, work):
    """The float64 form against the float64 arithmetic bound: the FMA probe's
    rate in FLOP/s and, since DADD and DMUL take a float64 pipe slot like DFMA,
    in float64 instructions per second (probe TFLOP/s / 2)."""
    if fp64_peak and work:
        flops, instr = work
        cells_s = r["mlups"] * 1e6
        r["fp64_alu"] = {"bound": "alu", "flops_per_cell": flops, "achieved_tflops": flops * cells_s / 1e12,
                         "peak_tflops": fp64_peak, "frac_flops": flops * cells_s / 1e12 / fp64_peak,
                         "fp64_instr_per_cell": instr, "achieved_ginstr_s": instr * cells_s / 1e9,
                         "peak_ginstr_s": fp64_peak / 2 * 1e3, "frac_pipe": instr * cells_s / 1e9 / (fp64_peak / 2 * 1e3),
                         "peak_source": "lbm_fp64_peak probe, same run"}


def _fp64_flops_per_cell(workload: str):
    """(float64 FLOP, float64 instructions) per cell update of a workload's step
    (ncu op counts, profiles/fp64_flops.txt)."""
    path = os.path.join(ROOT, "profiles", "fp64_flops.txt")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == workload:
                return float(parts[1]), float(parts[2])
    return None


def _first_step(lbm, newton_case, mlp_case, params):
    """Pass times of the first step after lbm_init, whose Newton guess is the
    initial temperature field, against the learned start (same kernel: the
    autotuned one)."""
    out = {}
    for name, case, p in (("newton_from_initial_T", newton_case, None), ("learned_start", mlp_case, params)):
        sim = lbm.Simulation(case)
        if p is not None:
            lbm.lbm_mlp_load(sim.h, p)
        sim.init()
        sim.autotune(2)  # restores the initial state
        out[name] = _pass_times(lbm, sim, 1)
        sim.close()
    return out


# the workloads of the forms, with the lattice-unit rescaling of the paper's constants that
# stability on the oracle forced (named so that each line says what it ran)
_FORM_WORKLOADS = (
    ("pr_droplet_384", "3-D Peng-Robinson droplet 384^3 periodic: PR at 1/20 of the slab's temperature scale "
                       "(Tc 0.025, Pc 0.00768503, kappa 0.01, Q 2.5e-8), eta/mu 10, radius 48, T/Tc 0.9, central Phi"),
    ("vdw_512", "2-D van der Waals quench 512^2 periodic: a = 9/245 (the paper's 9/49 x 0.2), b = 2/21, kappa 0.02, "
                "g = 2e-7 (the paper's 1e-6 x 0.2), eta/mu 3, T/Tc 0.9, rho mid-Maxwell + 1 % noise, central Phi"),
    ("vdw_4096", "the same fluid and recipe as the 512^2 quench on 4096^2"),
    ("vdw_batch_64", "64 independent 2-D van der Waals quenches, sides log-uniform 64-1024 rounded to multiples "
                     "of 8 (seed 4), T/Tc uniform 0.8-0.98, the 512^2 quench's rescaled fluid"),
    ("pr_slab_256", "3-D Peng-Robinson heated slab 256^3, walls in z: Tc 0.5, Pc 0.1537005, omega 0.1, kappa 0.2, "
                    "g = 1e-5, Q = 1e-6 in the bottom 10 % of z, T/Tc 0.95 + 0.1 % noise, upwind-biased Phi"),
    ("thermal_couette", "3-D thermal Couette 256 x 256 x 128 between extrapolation walls, ideal gas, Pr 2, central Phi"),
    ("fanno_duct", "bundle of 128 x 128 periodic ducts of 256 cells, total-state inlet, pressure outlet, "
                   "friction, ideal gas at Ma 0.3, central Phi"),
    ("ideal_2d_128", "2-D ideal gas 128^2: acoustic pulse and shear wave, F_x 1e-5, Q 1e-6, upwind-biased Phi"),
)


def _measure_forms(lbm, wl, torch, steps, headline=None):
    """Every form on its full-size workload (few steps each), next to the
    plain float64 GPU path of the same workload: MLUPS, HBM fraction, speed-up
    and deviation from float64 after the same steps."""
    res = {}
    try:
        fp64_peak, _ = lbm.lbm_fp64_peak()
        res["fp64_fma_peak_tflops"] = fp64_peak
    except Exception as e:
        fp64_peak = None
        res["fp64_fma_peak_tflops"] = f"unavailable: {e}"
    try:
        nd = max(4, steps // 2)
        # 3-D droplet (the headline workload): float64 beside it, and the learned temperature start
        d64, fd64 = _form(lbm, torch, wl.pr_droplet(384, storage="f64"), nd, 8, warm=1, passes=True)
        _fp64_bound(d64, fp64_peak, _fp64_flops_per_cell("pr_droplet_384_f64"))
        res["f64_pr_droplet_384_newton"] = d64
        torch.cuda.empty_cache()
        drop = wl.pr_droplet(384, storage="f32")
        newton, fdn = _form(lbm, torch, drop, nd, 4, warm=1, passes=True)
        _vs_f64(d64, fd64, newton, fdn)
        res["f32_pr_droplet_384_newton"] = newton
        le = lbm.structs_from_case(drop)[1]
        params = np.zeros(lbm.lbm_mlp_nparams(), dtype=np.float32)
        t0 = time.perf_counter()
        lbm.lbm_mlp_train(le, (0.1, 2.6, 0.85, 1.05), 1_000_000, 2000, 1024, 2e-3, 7, True, params)
        train_s = time.perf_counter() - t0
        drop_m = wl.pr_droplet(384, storage="f32")
        drop_m.t_solver = 1
        r, fr = _form(lbm, torch, drop_m, nd, 4, mlp=params, warm=1, passes=True)
        _vs_f64(d64, fd64, r, fr)
        r["train_s"] = train_s
        r["speedup_vs_f32_newton"] = newton["ms_per_step"] / r["ms_per_step"]
        r["rel_dev_vs_f32_newton"] = {"rho": _rel_dev(fr[0], fdn[0]), "T": _rel_dev(fr[1], fdn[1])}
        # cells whose learned temperature met the Newton tolerance in its first correction
        r["learned_start_accept_frac"] = 1.0 - r["diagnostics"][3] / float(r["cells"] * r["steps_since_init"])
        # the first step after lbm_init: Newton from the initial temperature field against T_hat
        r["first_step_after_init"] = _first_step(lbm, drop, drop_m, params)
        r["first_step_after_init"]["speedup_of_macroscopic_pass"] = (
            r["first_step_after_init"]["newton_from_initial_T"]["pass1_ms"] /
            r["first_step_after_init"]["learned_start"]["pass1_ms"])
        res["f32_pr_droplet_384_mlp"] = r
        del fd64
        torch.cuda.empty_cache()
        # the 512^2 van der Waals quench (the 2-D fused kernel), float64 beside it
        r64, f64 = _form(lbm, torch, wl.vdw_spinodal(512, storage="f64"), steps, 8, warm=0)
        _fp64_bound(r64, fp64_peak, _fp64_flops_per_cell("vdw_spinodal_512_f64"))
        res["f64_vdw_512"] = r64
        r, fr = _form(lbm, torch, wl.vdw_spinodal(512, storage="f32"), steps, 4, warm=0)
        _vs_f64(r64, f64, r, fr)
        traffic, ncu_us = _ncu_traffic("k_fused", "vdw_spinodal_512_f32")
        r["ncu_dram_bytes_per_launch"] = traffic
        res["f32_vdw_512"] = r
        # the isothermal mode (f only; algorithmic bytes 2 Q s) beside the full model
        iso = wl.vdw_spinodal(512, storage="f32")
        iso.isothermal = 1
        ri, _ = _form(lbm, torch, iso, steps, 4, warm=0, pops=1)
        ri["speedup_vs_full_model"] = r["ms_per_step"] / ri["ms_per_step"]
        res["f32_vdw_512_isothermal"] = ri
        # a 4096^2 quench (2.4 GB of float32 populations, far above L2): the 2-D row march
        r, fr = _form(lbm, torch, wl.vdw_spinodal(4096, storage="f32"), steps, 4, warm=0)
        traffic, ncu_us = _ncu_traffic("k_ymarch", "vdw_spinodal_4096_f32")
        r["ncu_dram_bytes_per_launch"] = traffic
        res["f32_vdw_4096"] = r
        rb, _ = _form(lbm, torch, wl.vdw_spinodal(4096, storage="bf16"), steps, 2, warm=0)
        rb["speedup_vs_f32"] = r["ms_per_step"] / rb["ms_per_step"]
        res["bf16_vdw_4096"] = rb
        torch.cuda.empty_cache()
        # 64 simulations per launch under CUDA graphs
        b64, fb64 = _form(lbm, torch, wl.vdw_batch(64, storage="f64"), steps, 8, graphs=10, warm=0)
        res["f64_vdw_batch_64"] = b64
        r, fr = _form(lbm, torch, wl.vdw_batch(64, storage="f32"), steps, 4, graphs=10, warm=0)
        _vs_f64(b64, fb64, r, fr)
        res["f32_vdw_batch_64"] = r
        torch.cuda.empty_cache()
        # 3-D heated slab: float64, float32, and 16-bit storage with offsets
        s64, fs64 = _form(lbm, torch, wl.pr_heated_slab(256, storage="f64"), steps, 8, warm=0, passes=True)
        _fp64_bound(s64, fp64_peak, _fp64_flops_per_cell("pr_heated_slab_256_f64"))
        res["f64_pr_slab_256"] = s64
        for st, sb in (("f32", 4), ("bf16", 2), ("f16", 2)):
            r, fr = _form(lbm, torch, wl.pr_heated_slab(256, storage=st), steps, sb, warm=0, passes=True)
            _vs_f64(s64, fs64, r, fr)
            res[f"{st}_pr_slab_256"] = r
        res["bf16_pr_slab_256"]["speedup_vs_f32"] = (res["f32_pr_slab_256"]["ms_per_step"] /
                                                     res["bf16_pr_slab_256"]["ms_per_step"])
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
        # extrapolation walls (z-march) and a friction duct: thermal Couette, Fanno duct
        res["f32_thermal_couette_256x256x128"], _ = _form(lbm, torch, wl.thermal_couette(256, 128),
                                                               steps, 4, tune=False, warm=2)
        res["f32_fanno_duct_128x128x256"], _ = _form(lbm, torch, wl.fanno_duct(128, 256), steps, 4,
                                                          tune=False, warm=2)
        r, _ = _form(lbm, torch, wl.acoustic_shear(128, storage="f64"), steps, 8)
        res["f64_ideal_2d_128"] = r
        torch.cuda.empty_cache()
    except Exception as e:  # report what was measured
        res["error"] = f"{type(e).__name__}: {e}"
    for key, val in res.items():
        if isinstance(val, dict):
            for part, desc in _FORM_WORKLOADS:
                if part in key:
                    val["workload"] = desc
                    break
    return res


def run_reference(args):
    """The FP64 CPU oracle on the headline workload: each step is one time
    step of a bounded sample of it (a 96^3 window of the 384^3 droplet)."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from oracle import oracle as orc
    from paper_2609_28679_b300 import workloads as wl

    case = wl.pr_droplet(384, storage="f64")
    sub, fields = _oracle_window(case, 48)
    o = orc.Oracle(orc.params_from_case(sub))
    o.init(*fields)
    o.step(max(args.warmup, 1))
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = sub.ncell * args.steps / dt / 1e6
    cores = orc.get_threads()
    sample = (f"{args.steps} time steps of the 96^3 periodic window of the 384^3 droplet centred on its interface "
              f"({sub.ncell} cells; FP64 C oracle, OpenMP)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": HEADLINE_DESC, "cells": case.ncell},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
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
    case = wl.pr_droplet(384, storage="f32")
    sim = lbm.Simulation(case)
    sim.init()
    if args.kernel == "auto":
        # warm-up includes the autotuner (kernel variant and tile for this workload; state restored)
        sim.autotune(3)
    else:
        kind, _, tile = args.kernel.partition(":")
        names = {"fused": lbm.LBM_KERNEL_FUSED, "split": lbm.LBM_KERNEL_SPLIT, "zmarch": lbm.LBM_KERNEL_ZMARCH,
                 "zgather": lbm.LBM_KERNEL_ZGATHER}
        t = [int(v) for v in tile.split("x")] if tile else [0, 0, 0]
        lbm.lbm_set_kernel(sim.h, names[kind], *(t + [0] * (3 - len(t))))
    variant, tx, ty, tz = sim.kernel()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        sim.step(1)
    torch.cuda.synchronize()

    # device-timed region: K eager steps between two events on the launching stream; the
    # populations (24.5 GB) are far larger than L2, so no flush is needed between steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    total_ms = max_over_ranks(e0.elapsed_time(e1))
    # the same steps again with events between the passes (the dominant kernel's own time)
    passes = _pass_times(lbm, sim, args.steps)
    diag = sim.diagnostics()

    # end to end through the C ABI with host buffers: upload the state, one step, read the fields back
    # (float32 fields for the float32 simulation: lbm_init_f32 / lbm_moments_f32)
    rho, u, T = case.fields()
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).pin_memory().numpy()
    rho_h, u_h, T_h = f32(rho), f32(u), f32(T)
    out_r = torch.empty(case.ncell, dtype=torch.float32).pin_memory().numpy()
    out_u = torch.empty(3 * case.ncell, dtype=torch.float32).pin_memory().numpy()
    out_T = torch.empty(case.ncell, dtype=torch.float32).pin_memory().numpy()
    e2e_steps = 3
    lbm.lbm_init_f32(sim.h, rho_h, u_h, T_h, 0)
    lbm.lbm_step(sim.h, 1)
    lbm.lbm_moments_f32(sim.h, out_r, out_u, out_T, 0)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(e2e_steps):
        lbm.lbm_init_f32(sim.h, rho_h, u_h, T_h, 0)
        lbm.lbm_step(sim.h, 1)
        lbm.lbm_moments_f32(sim.h, out_r, out_u, out_T, 0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    sim.close()
    del rho_h, u_h, T_h, out_r, out_u, out_T
    torch.cuda.empty_cache()

    forms = None
    if not args.no_forms:
        forms = _measure_forms(lbm, wl, torch, min(args.steps, 20))

    Q = 27
    alg_bytes = 4 * Q * 4 * case.ncell  # read + write f and g once, float32
    avg_ms = total_ms / args.steps
    peak, peak_src = _peaks()
    names = {lbm.LBM_KERNEL_FUSED: "k_fused", lbm.LBM_KERNEL_ZGATHER: "k_zgather", lbm.LBM_KERNEL_ZMARCH: "k_zmarch",
             lbm.LBM_KERNEL_SPLIT: "k_collide"}
    kname = names.get(variant, "k_collide")
    dom_ms = passes["pass3_ms"]  # the collide-stream pass: the dominant kernel of the step
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9
    value = aggregate_mlups(case.ncell, args.steps, world, total_ms)
    traffic, ncu_us = _ncu_traffic(kname, "pr_droplet_384_f32")
    launches_per_step = {lbm.LBM_KERNEL_FUSED: 1, lbm.LBM_KERNEL_SPLIT: 3}.get(variant, 2)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cb_case = wl.pr_droplet(384, storage="f64")
            cv, n, dt, cores, what = _oracle_mlups(cb_case, 20.0)
            cv1, n1, dt1, _, _ = _oracle_mlups(cb_case, 8.0, threads=1, half=24)
            _oracle_threads(cores)
            cpu = {"value": cv, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{n} time steps of a {what} ({dt:.1f} s, FP64 C oracle, OpenMP)",
                   "single_core": {"value": cv1, "unit": UNIT,
                                   "sample": f"{n1} time steps of a 48^3 window ({dt1:.1f} s)"},
                   "cpu_model": _cpu_model(), "nproc": os.cpu_count()}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; paper-shaped Peng-Robinson droplet)",
            "config": {"workload": HEADLINE_DESC, "cells": case.ncell, "storage": "f32",
                       "kernel": kname, "tile": [tx, ty, tz],
                       "l2": "not flushed: inputs larger than L2 (24.5 GB of populations per step)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": kname, "launch_ms": dom_ms,
                         "peak_source": peak_src,
                         "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "step_frac": alg_bytes / (avg_ms * 1e-3) / 1e9 / peak,
                         "ncu_dram_gbs": (traffic / (ncu_us * 1e-6) / 1e9) if traffic and ncu_us else None},
            "passes": {"macroscopic_ms": passes["pass1_ms"], "boundary_ms": passes["pass2_ms"],
                       "collide_stream_ms": passes["pass3_ms"], "step_ms": passes["step_ms"]},
            "e2e": {"value": case.ncell * e2e_steps / e2e_s / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": int(case.ncell * 5 * 4), "d2h_bytes_per_step": int(case.ncell * 5 * 4),
                    "what": "lbm_init_f32 from pinned float32 host fields (rho, u, T) + lbm_step(1) + "
                            "lbm_moments_f32 to pinned host"},
            "gpu_launches": args.steps * launches_per_step,
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the per-form measurements")
    ap.add_argument("--kernel", default="auto",
                    help="auto (autotuned), split, fused:TXxTY[xTZ], zmarch:TXxTYxZL or zgather:30x14xZL (pinned)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
