"""Build step of the CUDA library: nvcc, sm_103a only, one object per
translation unit compiled in parallel, linked into libfpgb300.so in-tree."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfpgb300.so")
LIB_CHECK = os.path.join(HERE, "libfpgb300_check.so")
SOURCES = ["api.cu", "pipe.cu", "metrics.cu", "cfl.cu", "probe.cu", "sweep_f32.cu", "sweep_f32_fix.cu", "sweep_f32_fix2.cu",
           "sweep_f32_bnd.cu", "sweep_f32_bnd_fix.cu", "sweep_f32_bnd_fix2.cu", "sweep_f64.cu", "sweep_f64_fix.cu",
           "sweep_f64_bnd.cu", "sweep_f64_bnd_fix.cu"]
HEADERS = ["fp_internal.h", "sweep.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [
        os.path.join(HERE, "..", "include", "fp.h")]
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=(), check: bool = False) -> str:
    """Compile and link the library; check=True builds the bounds-checking variant
    libfpgb300_check.so (-DFPK_BOUNDS_CHECK, objects in _build_check) beside it."""
    bdir = BUILD + "_check" if check else BUILD
    lib = LIB_CHECK if check else LIB
    extra = [*extra, "-DFPK_BOUNDS_CHECK"] if check else list(extra)
    os.makedirs(bdir, exist_ok=True)
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        if force or _stale(o, s):
            jobs.append([nvcc(), *ARCH, *FLAGS, *extra, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.returncode

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        rcs = list(ex.map(run, jobs))
    if any(rcs):
        raise RuntimeError("nvcc failed")
    objs = [os.path.join(bdir, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(lib):
        cmd = [nvcc(), *ARCH, "-shared", "-o", lib, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, check="--check" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
