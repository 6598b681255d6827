"""Build the CUDA library ``libjz.so`` in-tree for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then
linked into ``paper_2003_09926_gb300/libjz.so``.  No cmake, no torch
extension machinery: the library exposes a plain C ABI (``include/jz.h``).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libjz.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object, extra defines): the FP32 vector-record stage kernel is
# built once per tile shape the autotuner may choose
SOURCES = [(s, s.replace(".cu", ".o"), []) for s in
           ("jz_api.cu", "jz_grid.cu", "jz_reduce.cu", "jz_stage.cu", "jz_static.cu", "jz_peak.cu", "jz_stats.cu")]
SOURCES += [("jz_stage_v.cu", f"jz_stage_v_{ti}x{tj}.o", [f"-DVR_TI={ti}", f"-DVR_TJ={tj}"])
            for ti, tj in ((32, 16), (16, 32), (16, 16))]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps_newer(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "jz.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(entry, verbose: bool) -> str:
    src, objname, defines = entry
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, objname)
    if not _deps_newer(obj, path):
        return obj
    # host code: no fused multiply-add contraction (results that the host
    # forms, such as the statistics' rms, then round as plainly written)
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
           *defines, "-c", path, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
