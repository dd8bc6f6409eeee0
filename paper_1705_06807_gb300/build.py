"""Builds the CUDA library libparrep.so in-tree for sm_103a with nvcc.

The translation units are compiled in parallel; parrep_kernels.cu is compiled
once per part (-DPARREP_PART=0..11: the small kernels, then the run, batch and
serve kernels in each of the binary64, binary32 staged and binary32 direct
forms, and the batch and serve kernels in the mixed binary32 form), since each
persistent kernel inlines the whole of Algorithm 1.  Arithmetic contraction is off (-fmad=false) so that
the binary64/binary32 propensity and selection expressions round exactly as
written.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libparrep.so")
KERNEL_PARTS = 12
SOURCES = [("parrep_kernels.cu", i) for i in range(KERNEL_PARTS)] + [
    (f, None) for f in ["parrep_api.cu", "parrep_batch.cu", "parrep_serve.cu", "parrep_noalloc.cu", "parrep_uq.cu"]]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def flags(verbose_ptxas: bool = False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "parrep.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    fl = flags(verbose_ptxas)
    tag = f"{os.getpid()}"

    def compile_one(item):
        src, part = item
        stem = src.replace(".cu", "" if part is None else f".part{part}")
        obj = os.path.join(OUT_DIR, f"{stem}.{tag}.o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + fl
        if part is not None:
            cmd += [f"-DPARREP_PART={part}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose_ptxas:
            sys.stderr.write(r.stderr)
        return obj

    # the binary32 staged run / batch / serve parts take longest: start them first
    order = sorted(SOURCES, key=lambda it: (0 if it[1] in (10, 11, 2, 5, 8) else 1 if it[1] else 2))
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, order))
    tmp = LIB + f".{tag}.tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
