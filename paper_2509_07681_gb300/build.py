"""Builds ``libfuncsne.so`` (the C ABI of include/funcsne.h) for sm_103a with
nvcc: one object per translation unit, compiled in parallel, then linked.

``build(checked=True)`` builds ``libfuncsne_checked.so`` from the same
sources with -DFUNCSNE_CHECKED: the iteration kernels range-check every
point index they read from memory before using it to address a row or a
list, set the device error bit kErrIndex on a bad one and keep the access in
bounds. Select it with FUNCSNE_LIBRARY=<path> (see funcsne.load)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfuncsne.so")
LIB_CHECKED = os.path.join(HERE, "libfuncsne_checked.so")
SOURCES = ["api.cu", "init_kernels.cu", "insert_kernels.cu", "knn_exact.cu", "knn_noalloc.cu", "live_kernels.cu",
           "mlp_kernels.cu", "update_kernel.cu",
           "step_f32.cu", "step_bf16.cu", "step_fp8.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfuncsne.so")


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "funcsne.h"))
    return files


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the library (checked: the range-checked variant) if it is
    missing or older than its sources. Returns its path."""
    return build_many([checked], force=force, verbose=verbose)[0]


def build_many(variants, force: bool = False, verbose: bool = False) -> list[str]:
    """Compile several variants (False: the library, True: the range-checked
    one), all translation units in one parallel pool."""
    libs = [LIB_CHECKED if v else LIB for v in variants]
    todo = [v for v, lib in zip(variants, libs) if force or _stale(lib)]
    if not todo:
        return libs
    nvcc = _nvcc()

    def compile_one(job) -> str:
        src, checked = job
        out_dir = os.path.join(BUILD, "checked" if checked else "plain")
        os.makedirs(out_dir, exist_ok=True)
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *(["-DFUNCSNE_CHECKED"] if checked else []), "-c", os.path.join(CSRC, src),
               "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    jobs = [(src, v) for v in todo for src in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 8)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, v in enumerate(todo):
        lib = LIB_CHECKED if v else LIB
        tmp = lib + f".tmp{os.getpid()}"
        mine = objs[k * len(SOURCES):(k + 1) * len(SOURCES)]
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *mine]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return libs


if __name__ == "__main__":
    print(build_many([False, True], force=True, verbose=True))
