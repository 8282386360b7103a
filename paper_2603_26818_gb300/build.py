"""Compile the CUDA library libpfc.so (sm_103a) in-tree with nvcc.

One translation unit holds the pass kernels and the C ABI of include/pfc.h; the vendor cuFFT
plain-step baseline is a separate library, libpfc_cufft_baseline.so, so the product library
does not link cuFFT. Both are built in parallel.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpfc.so")
BASELINE_LIB = os.path.join(HERE, "libpfc_cufft_baseline.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpfc.so")
    return cand


def _sources(names):
    return [os.path.join(CSRC, n) for n in names]


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _deps():
    inc = os.path.join(os.path.dirname(HERE), "include", "pfc.h")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [inc]


def _compile(out, srcs, extra):
    cmd = [_nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-o", out + ".tmp", *srcs, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(out)}:\n{r.stderr[-4000:]}")
    os.replace(out + ".tmp", out)


def build(force: bool = False) -> str:
    deps = _deps()
    jobs = []
    if force or _stale(LIB, deps):
        jobs.append((LIB, _sources(["pfc_api.cu"]), []))
    if force or _stale(BASELINE_LIB, deps):
        jobs.append((BASELINE_LIB, _sources(["cufft_baseline.cu"]), ["-lcufft"]))
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(lambda j: _compile(*j), jobs))
    return LIB


if __name__ == "__main__":
    build(force=True)
    print(LIB)
