"""Build libniv.so in-tree with nvcc for sm_103a (one object per .cu, compiled in parallel)."""
import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libniv.so")
# Measurement aids that only the benchmark loads, kept out of the product library.
BENCH_CSRC = os.path.join(PKG, "bench_csrc")
BENCH_LIB = os.path.join(PKG, "libniv_peaks.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-DNIV_BUILD"]
# Extra compiler flags (e.g. kernel tuning defines); empty by default.
EXTRA = os.environ.get("NIV_NVCC_EXTRA", "").split()


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, inputs):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(i) > t for i in inputs)


def _compile(src, extra=()):
    prefix = "bench_" if os.path.dirname(src) == BENCH_CSRC else ""
    obj = os.path.join(BUILD, prefix + os.path.basename(src)[:-3] + ".o")
    if _stale(obj, [src] + _deps()):
        cmd = [NVCC, *ARCH, *FLAGS, *EXTRA, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj


def build(force=False, verbose_ptxas=False):
    """Compile every kernel source and link libniv.so next to this file; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for o in glob.glob(os.path.join(BUILD, "*.o")):
            os.remove(o)
    extra = ("-Xptxas", "-v") if verbose_ptxas else ()
    srcs = _sources()
    bench_srcs = sorted(glob.glob(os.path.join(BENCH_CSRC, "*.cu")))
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs) + len(bench_srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs + bench_srcs))
    for lib, lib_objs in ((LIB, objs[:len(srcs)]), (BENCH_LIB, objs[len(srcs):])):
        if lib_objs and (force or _stale(lib, lib_objs)):
            tmp = lib + ".tmp%d" % os.getpid()
            cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *lib_objs,
                   "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build())
