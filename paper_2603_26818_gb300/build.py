"""Compile the CUDA library libpfc.so (sm_103a) in-tree with nvcc.

Several translation units hold the pass kernels and the C ABI of include/pfc.h; the vendor cuFFT
plain-step baseline is a separate library, libpfc_cufft_baseline.so, so the product library
does not link cuFFT, and the FMA-rate probe used by the bench is a third, libpfc_probe.so. All
are built in parallel.
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
PROBE_LIB = os.path.join(HERE, "libpfc_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpfc.so")
    return cand


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _deps():
    inc = os.path.join(os.path.dirname(HERE), "include", "pfc.h")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [inc]


def _run(cmd, what):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {what}:\n{r.stderr[-4000:]}")


def _compile_obj(src, obj):
    _run([_nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
          "-o", obj, src], os.path.basename(src))


def _link(out, objs, extra):
    _run([_nvcc(), *ARCH, "-shared", "-o", out + ".tmp", *objs, *extra], os.path.basename(out))
    os.replace(out + ".tmp", out)


# translation units of libpfc.so: host plan logic, the kernels of each precision, and the
# allocation-free step, the persistent batch kernel of each precision, the amplitude-expansion model
LIB_UNITS = ["pfc_api.cu", "pfc_batch.cu", "pfc_kern_f32.cu", "pfc_kern_f64.cu", "pfc_line_fixed_f32.cu",
             "pfc_line_fixed_f64.cu", "pfc_row_fixed_f32.cu", "pfc_row_fixed_f64.cu", "pfc_noalloc.cu",
             "pfc_persist_f32_128.cu", "pfc_persist_f32_256.cu", "pfc_persist_f32_512.cu",
             "pfc_persist_f64_128.cu", "pfc_persist_f64_256.cu", "pfc_persist_f64_512.cu", "pfc_apfc.cu"]


def build(force: bool = False) -> str:
    deps = _deps()
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    jobs = []
    objs = []
    for u in LIB_UNITS:
        obj = os.path.join(objdir, u.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, deps):
            jobs.append((os.path.join(CSRC, u), obj))
    base_obj = os.path.join(objdir, "cufft_baseline.o")
    if force or _stale(base_obj, deps):
        jobs.append((os.path.join(CSRC, "cufft_baseline.cu"), base_obj))
    probe_obj = os.path.join(objdir, "peak_probe.o")
    if force or _stale(probe_obj, deps):
        jobs.append((os.path.join(CSRC, "peak_probe.cu"), probe_obj))
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(lambda j: _compile_obj(*j), jobs))
    if force or jobs or not os.path.exists(LIB):
        _link(LIB, objs, [])
    if force or jobs or not os.path.exists(BASELINE_LIB):
        _link(BASELINE_LIB, [base_obj], ["-lcufft"])
    if force or jobs or not os.path.exists(PROBE_LIB):
        _link(PROBE_LIB, [probe_obj], [])
    return LIB


if __name__ == "__main__":
    build(force=True)
    print(LIB)
