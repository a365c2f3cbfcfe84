"""Build the IBF CUDA library (sm_103a) in-tree with nvcc.

Produces ``paper_1605_03616_gb300/_build/libibf_gb300.so`` from the
translation units in ``csrc/``, compiled in parallel.  The construction unit
(``ibf_plan.cu``) is compiled with ``-fmad=false`` so that FP64 grid points and
phases round like a plain sequential evaluation of the paper's formulas.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libibf_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
          "--expt-relaxed-constexpr"]
UNITS = {
    "ibf_plan.cu": ["-fmad=false"],
    "ibf_explicit.cu": [],
    "ibf_fused_f32.cu": [],
    "ibf_fused_f64.cu": [],
    "ibf_static.cu": [],
    "ibf_batch.cu": [],
    "ibf_2d_build.cu": ["-fmad=false"],
    "ibf_2d_apply.cu": [],
    "ibf_optimal.cu": [],
    "ibf_amplitude.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the IBF library needs the CUDA toolkit to build")


def _sources_newer_than(path: str) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    for fn in os.listdir(CSRC):
        if os.path.getmtime(os.path.join(CSRC, fn)) > t:
            return True
    hdr = os.path.join(os.path.dirname(HERE), "include", "ibf.h")
    return os.path.getmtime(hdr) > t or os.path.getmtime(__file__) > t


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and not _sources_newer_than(LIB):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    extra = list(extra or [])

    def compile_one(unit: str) -> str:
        obj = os.path.join(OUT_DIR, unit.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *UNITS[unit], *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, res.stdout, res.stderr))
        if verbose and res.stderr:
            print(res.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s\n%s" % (res.stdout, res.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
