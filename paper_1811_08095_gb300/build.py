"""Build the in-tree CUDA library `libodwf.so` for sm_103a with nvcc (no cmake).

Every translation unit under csrc/ compiles in parallel; the objects link into
paper_1811_08095_gb300/libodwf.so next to this file.  Rebuilds only when a source
or header is newer than the library.  build(bounds_check=True) makes the debug variant
libodwf_check.so (ODWF_BOUNDS_CHECK: the kernels check every gathered index and the calls
report an out-of-range one as ODWF_ECUDA); both variants can be built in one call.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libodwf.so")
LIB_CHECK = os.path.join(HERE, "libodwf_check.so")
BUILD = os.path.join(HERE, "_build")
BUILD_CHECK = os.path.join(HERE, "_build_check")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libodwf.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(variants, verbose):
    """Compile and link every (library, object directory, extra flags) variant, all
    translation units of all variants in parallel."""
    nvcc = _nvcc()
    procs = []
    for lib, bdir, extra in variants:
        os.makedirs(bdir, exist_ok=True)
        for src in sources():
            obj = os.path.join(bdir, os.path.basename(src) + ".o")
            cmd = [nvcc] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [nvcc] + NVCC_FLAGS + extra + ["-x", "cu"] + ARCH + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        msg = "\n".join("%s:\n%s" % f for f in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    for lib, bdir, _ in variants:
        objs = [os.path.join(bdir, os.path.basename(src) + ".o") for src in sources()]
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs)
        os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    """Build libodwf.so (and libodwf_check.so when bounds_check) if stale; returns libodwf.so's path."""
    variants = []
    if force or _stale(LIB):
        variants.append((LIB, BUILD, []))
    if bounds_check and (force or _stale(LIB_CHECK)):
        variants.append((LIB_CHECK, BUILD_CHECK, ["-DODWF_BOUNDS_CHECK"]))
    if variants:
        _compile(variants, verbose)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, bounds_check="--bounds-check" in sys.argv))
