"""Build libmg5.so (sm_103a) in-tree with nvcc.

Every .cu file under csrc/ is compiled in parallel to an object file, then
linked into paper_1511_08200_gb300/libmg5.so with the CUDA runtime linked
statically (no rpath needed; torch and the library share the driver's primary
context, so torch streams and device pointers pass straight through).

`build(bounds=True)` (or `python -m paper_1511_08200_gb300._build --bounds`) makes the
range-checked variant libmg5_bounds.so (-DMG5_BOUNDS: every kernel's global and shared
element accesses checked against the known allocations, violations recorded in a device
error word instead of faulting); the binding loads it when MG5_BOUNDS=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build", platform.machine())   # objects per host architecture
LIB = os.path.join(PKG, "libmg5.so")
LIB_BOUNDS = os.path.join(PKG, "libmg5_bounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _needs(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, bounds: bool = False) -> str:
    obj_dir = OBJ + ("-bounds" if bounds else "")
    lib = LIB_BOUNDS if bounds else LIB
    extra = ["-DMG5_BOUNDS"] if bounds else []
    os.makedirs(obj_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "mg5.h")]
    jobs = []
    for s in srcs:
        o = os.path.join(obj_dir, os.path.basename(s)[:-3] + ".o")
        if force or _needs(o, [s] + hdrs):
            jobs.append((s, o))

    def compile_one(so):
        s, o = so
        cmd = [NVCC] + _flags() + extra + ["-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (s, r.stdout, r.stderr))
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for msg in ex.map(compile_one, jobs):
            if verbose and msg:
                print(msg, file=sys.stderr)
    objs = [os.path.join(obj_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    if force or jobs or not os.path.exists(lib) or _needs(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, bounds="--bounds" in sys.argv))
