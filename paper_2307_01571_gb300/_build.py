"""Compiles the CUDA library ``libkd.so`` in-tree for sm_103a.

The translation units (host API, the FP32 sweeps once per launch variant, the
double-word sweeps once per axis and shape, the FP64 sweeps, the tensor-core sweeps, the allocation-free entry and the MLP kernels) compile in parallel with nvcc; the
CUDA runtime is linked statically so the library only needs the driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkd.so")
SWEEP_VARIANTS = 4    # KD_SWEEP_VARIANTS in csrc/kd_internal.h
# (source, object, extra defines)
UNITS = ([("kd_api.cu", "kd_api.o", [])]
         + [("kd_sweep_f32.cu", f"kd_sweep_f32_v{v}.o", [f"-DKD_SWEEP_VARIANT={v}"])
            for v in range(SWEEP_VARIANTS)]
         + [("kd_sweep_dw.cu", f"kd_sweep_dw_p{p}.o", [f"-DKD_DW_PART={p}"]) for p in range(6)]
         + [("kd_sweep_f64.cu", "kd_sweep_f64.o", []), ("kd_tc.cu", "kd_tc.o", []),
            ("kd_noalloc.cu", "kd_noalloc.o", []), ("kd_mlp.cu", "kd_mlp.o", []),
            ("kd_persist.cu", "kd_persist.o", [])])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         f"-I{os.path.join(ROOT, 'include')}"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkd.so")
    return p


def _inputs():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "kd.h"))
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(unit):
        src, obj, defs = unit
        obj = os.path.join(BUILD, obj)
        cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
