"""Run a few time steps of one synthetic workload on the GPU and print the
time per step: the command line that profilers wrap.

    python -m paper_2609_28679_b300.run_case vdw_spinodal 512 f32 fused:64x14
    python -m paper_2609_28679_b300.run_case pr_heated_slab 128 f32 zmarch:30x14x32 --steps 4

Workloads: acoustic_shear, vdw_spinodal, pr_heated_slab, pr_droplet (size =
cells per side), thermal_couette (n x n x n/2), fanno_duct (n x n x 2n).  Kernel: auto (autotuner), split, fused[:TXxTY[xTZ]] or
zmarch[:TXxTYxZL], zgather[:30x14xZL] or ymarch[:0xYL] (2-D).
"""
from __future__ import annotations

import argparse
import json
import sys

from . import lbm
from . import workloads as wl

_CASES = {
    "acoustic_shear": lambda n, st: wl.acoustic_shear(n, storage=st),
    "vdw_spinodal": lambda n, st: wl.vdw_spinodal(n, storage=st),
    "pr_heated_slab": lambda n, st: wl.pr_heated_slab(n, storage=st),
    "pr_droplet": lambda n, st: wl.pr_droplet(n, storage=st, radius=n / 8.0),
    "thermal_couette": lambda n, st: wl.thermal_couette(n, n // 2, storage=st),
    "fanno_duct": lambda n, st: wl.fanno_duct(n, 2 * n, storage=st),
}
_VARIANTS = {"split": lbm.LBM_KERNEL_SPLIT, "fused": lbm.LBM_KERNEL_FUSED, "zmarch": lbm.LBM_KERNEL_ZMARCH,
             "zgather": lbm.LBM_KERNEL_ZGATHER, "ymarch": lbm.LBM_KERNEL_YMARCH}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("workload", choices=sorted(_CASES))
    ap.add_argument("size", type=int)
    ap.add_argument("storage", choices=["f64", "f32", "bf16", "f16"])
    ap.add_argument("kernel", nargs="?", default="auto")
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=2)
    args = ap.parse_args(argv)

    import torch

    if not torch.cuda.is_available():
        raise SystemExit("run_case: no CUDA device (the library has no CPU path)")
    case = _CASES[args.workload](args.size, args.storage)
    sim = lbm.Simulation(case)
    sim.init()
    if args.kernel == "auto":
        sim.autotune(3)
    else:
        kind, _, tile = args.kernel.partition(":")
        t = [int(v) for v in tile.split("x")] if tile else []
        lbm.lbm_set_kernel(sim.h, _VARIANTS[kind], *(t + [0] * (3 - len(t))))
    sim.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sim.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    out = {"workload": case.name, "cells": case.ncell, "storage": args.storage, "kernel": list(sim.kernel()),
           "ms_per_step": ms, "mlups": case.ncell / (ms * 1e3), "diagnostics": [int(v) for v in sim.diagnostics()]}
    sim.close()
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
