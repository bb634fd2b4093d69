"""Builds the in-tree CUDA library ``_lib/libcp.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked with the CUDA
runtime.  No CMake, no torch extension machinery: the library has a plain
C ABI (include/cp.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libcp.so")
# instruction-rate probes (paper_1412_1840_gb300.peaks): a separate library, not part of the path
PROBE_SRC = os.path.join(CSRC, "probe", "cp_peaks.cu")
PROBE_LIB = os.path.join(OUT_DIR, "libcppeaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code keeps IEEE evaluation order (no FMA contraction), so FP64 decisions
# taken on the host match their definitions on any host architecture.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(ROOT, "include", "cp.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build_probe(force: bool = False) -> str:
    """Compiles the instruction-rate probes into their own library."""
    deps = [PROBE_SRC, os.path.join(CSRC, "cp_tc.cuh")]
    if not force and os.path.exists(PROBE_LIB) and all(os.path.getmtime(d) <= os.path.getmtime(PROBE_LIB) for d in deps):
        return PROBE_LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = PROBE_LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + FLAGS + ["-shared", "-cudart", "static", PROBE_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (PROBE_SRC, r.stdout, r.stderr))
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    with cf.ThreadPoolExecutor(max_workers=1) as ex:
        probe = ex.submit(build_probe, force)
        lib = _build_lib(force, verbose)
        probe.result()
    return lib


def _build_lib(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
