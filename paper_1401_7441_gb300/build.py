"""In-tree build of the sm_103a library ``liblsw.so`` (nvcc + the host compiler).

Six translation units compiled in parallel, one -gencode (sm_103a), static CUDA
runtime, no cmake.  Host code is compiled without floating-point contraction so that
the locreg membership tests and the filter derivation round exactly as specified.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
CHECKED = os.environ.get("LSW_CHECKED", "0") == "1"   # self-checking build (bounds on every access)
LIB = os.path.join(HERE, "liblsw_checked.so" if CHECKED else "liblsw.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (set NVCC or add /usr/local/cuda/bin to PATH)")


def sources():
    return [os.path.join(CSRC, f) for f in ("lsw_kernels.cu", "lsw_panels.cu", "lsw_foe.cu", "lsw_confine.cu", "lsw_host.cpp", "lsw_filters.cpp")]


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile (if stale) and return the path of liblsw.so."""
    srcs = sources()
    deps = srcs + [os.path.join(CSRC, "lsw_internal.h"), os.path.join(CSRC, "lsw_device.h"), os.path.join(CSRC, "lsw_tc.h"), os.path.join(ROOT, "include", "lsw.h"),
                   os.path.abspath(__file__)]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    build_dir = BUILD + ("_checked" if CHECKED else "")
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    host_flags = "-fPIC,-O2,-ffp-contract=off,-fno-fast-math"
    procs = []
    objs = []
    for src in srcs:
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", ARCH, "-lineinfo",
               "-Xcompiler", host_flags, "--fmad=true", "-diag-suppress=177"] + inc + (["-DLSW_CHECKED"] if CHECKED else []) \
            + os.environ.get("LSW_NVCC_DEFINES", "").split()
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "c++", "-c", src, "-o", obj, "-std=c++17", "-Xcompiler", host_flags] + inc
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out.decode())
        if p.returncode != 0:
            failed.append((cmd, out.decode()))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("liblsw build failed:\n" + msg)
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp, *objs, ARCH, "-cudart", "static", "-Xcompiler", "-fPIC", "-lpthread"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("liblsw link failed:\n" + r.stdout.decode())
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
