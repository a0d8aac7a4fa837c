"""Build the in-tree CUDA library ``liblbm.so`` for sm_103a.

nvcc compiles the kernels and the C ABI; g++ compiles the small glue that
takes device memory and the current stream from PyTorch's libc10_cuda.  The
shared CUDA runtime is the one PyTorch loads (same soname), so streams and
allocations are shared with the caller's tensors.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbm.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _torch_dirs():
    import torch  # noqa: F401  (only to locate headers and libraries)

    tdir = os.path.dirname(torch.__file__)
    cu = os.path.join(os.path.dirname(tdir), "nvidia", "cu13", "lib")
    return os.path.join(tdir, "include"), os.path.join(tdir, "lib"), cu, int(torch._C._GLIBCXX_USE_CXX11_ABI)


def _newer(target: str, sources) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    tinc, tlib, cudart_dir, abi = _torch_dirs()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    objs, jobs = [], []
    for cu in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        obj = os.path.join(BUILD, os.path.basename(cu) + ".o")
        if force or _newer(obj, [cu] + headers):
            cmd = ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-prec-div=false", "-prec-sqrt=false",
                   "-Xcompiler", "-fPIC", "-cudart", "shared",
                   "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-c", cu, "-o", obj]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
        objs.append(obj)
    if jobs:
        from concurrent.futures import ThreadPoolExecutor

        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda c: _run(c, verbose), jobs))
    glue = os.path.join(CSRC, "lbm_glue.cpp")
    gobj = os.path.join(BUILD, "lbm_glue.cpp.o")
    if force or _newer(gobj, [glue]):
        _run(["g++", "-O2", "-fPIC", "-std=c++17", f"-D_GLIBCXX_USE_CXX11_ABI={abi}", "-I", tinc,
              "-I", os.path.join(cuda, "include"), "-c", glue, "-o", gobj], verbose)
    objs.append(gobj)
    if force or _newer(LIB, objs):
        _run(["nvcc", ARCH, "-shared", "-cudart", "shared", "-o", LIB] + objs +
             ["-L", tlib, "-lc10", "-lc10_cuda", "-L", cudart_dir, "-L", os.path.join(cuda, "lib64"),
              "-Xlinker", f"-rpath,{tlib}", "-Xlinker", f"-rpath,{cudart_dir}",
              "-Xlinker", f"-rpath,{os.path.join(cuda, 'lib64')}"], verbose)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv)
