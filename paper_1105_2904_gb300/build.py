"""Builds the CUDA library ``liblbmp.so`` in-tree for sm_103a (GB300).

Eleven translation units are compiled in parallel with nvcc, one ``-gencode`` each:
``api.cu`` (host C-ABI; host code with -ffp-contract=off), ``sweep_f64.cu`` and
``particles.cu`` (-fmad=false: FP64 arithmetic evaluated exactly as written),
``sweep_f32.cu``, ``sweep_f16.cu``, ``sweep_bf16.cu`` (FP32 / FP16 / BF16 storage),
``noalloc.cu`` (the allocation-free boundary-site exchange), ``batch.cu`` (batched
ensembles), ``mlp.cu`` (the closure network), ``checkpoint.cu`` (checkpoint and resume),
``diag.cu`` (state diagnostics, -fmad=false).
Output: ``paper_1105_2904_gb300/_lib/``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
SO = os.path.join(LIBDIR, "liblbmp.so")
# The bounds-checked build (-DLBM_DEBUG): kernels check particle ids, record slots and
# contact-list indices and report LBM_E_BOUNDS through the device status word instead of
# reading or writing out of range. Built on request only; lbmp loads it when LBMP_DEBUG=1.
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
SO_DEBUG = os.path.join(PKG, "_lib_debug", "liblbmp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-I", INCLUDE, "-I", CSRC]
UNITS = {
    "api.cu": [],
    "sweep_f64.cu": ["-fmad=false"],
    "particles.cu": ["-fmad=false"],
    "sweep_f32.cu": [],
    "sweep_f16.cu": [],
    "sweep_bf16.cu": [],
    "noalloc.cu": [],
    "batch.cu": [],
    "mlp.cu": [],
    "checkpoint.cu": [],
    "diag.cu": ["-fmad=false"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbmp.h"),
                                                                os.path.abspath(__file__)]


def up_to_date(so: str = SO) -> bool:
    if not os.path.exists(so):
        return False
    t = os.path.getmtime(so)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, debug=None) -> str:
    """Builds liblbmp.so (debug=True: the bounds-checked build, SO_DEBUG; None: the build the
    binding loads, i.e. the bounds-checked one when LBMP_DEBUG=1)."""
    if debug is None:
        debug = os.environ.get("LBMP_DEBUG") == "1"
    so = SO_DEBUG if debug else SO
    objdir = BUILD_DEBUG if debug else BUILD
    if not force and up_to_date(so):
        return so
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(os.path.dirname(so), exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(objdir, unit.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc] + ARCH + COMMON + extra + (["-DLBM_DEBUG"] if debug else []) + \
            ["-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((unit, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for unit, cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(unit)
    if failed:
        raise RuntimeError("nvcc failed for %s" % ", ".join(failed))
    tmp = so + ".%d.tmp" % os.getpid()
    subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug=True if "--debug" in sys.argv else None))
