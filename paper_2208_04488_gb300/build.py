"""Build the in-tree CUDA library ``_build/libhrm.so`` for sm_103a with nvcc.

Each translation unit compiles in parallel. The per-cell unit, the FP64
per-midpoint units and the precision form's units are built without FMA
contraction: the FP64 path evaluates every expression in the order written with
IEEE rounding, and the precision form's FP32 expressions round the same way in
every kernel that inlines them (its FMAs are explicit fma()/fmaf() calls).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
# HRM_BOUNDS_CHECK=1: the bounds-check build (index checks in the kernels, see
# hrm_bounds_violations) into its own folder
BOUNDS_CHECK = os.environ.get("HRM_BOUNDS_CHECK", "0") == "1"
OUT = os.path.join(HERE, "_build_check" if BOUNDS_CHECK else "_build")
LIB = os.path.join(OUT, "libhrm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code: no FP contraction either (species constants are derived on the host)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr"] + (["-DHRM_BOUNDS_CHECK"] if BOUNDS_CHECK else [])
UNITS = {
    "hrm_cell.cu": ["--fmad=false"],
    "hrm_face64_d1.cu": ["--fmad=false"],
    "hrm_face64_d2.cu": ["--fmad=false"],
    "hrm_face64_d3.cu": ["--fmad=false"],
    "hrm_face32_d1.cu": ["--fmad=false"],
    "hrm_face32_d2.cu": ["--fmad=false"],
    "hrm_face32_d3.cu": ["--fmad=false"],
    "hrm_api.cu": [],
    "hrm_probe.cu": [],
    "hrm_noalloc.cu": ["--fmad=false"],
    "hrm_batch64_d2.cu": ["--fmad=false"],
    "hrm_batch32_d2.cu": ["--fmad=false"],
    "hrm_batch_api.cu": [],
    "hrm_learned.cu": [],
    "hrm_learned_data.cu": ["--fmad=false"],
}


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "hrm.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(OUT, unit.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((unit, out.decode(errors="replace")))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {u}\n{o}" for u, o in failed))
    tmp = LIB + ".tmp"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
