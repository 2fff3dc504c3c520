"""Builds libnmc.so in-tree for sm_103a with nvcc (no cmake, no torch extension).

Each .cu file is compiled to an object in parallel, then linked into
paper_2601_00976_gb300/_lib/libnmc.so.  Objects are rebuilt when their source or
any header is newer.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libnmc.so")
# the NMC_DEBUG build (bounds checks that record a failed index in a device error word)
OUT_DEBUG = os.path.join(HERE, "_lib_debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, "libnmc.so")
# the NMC_TRACE build (per-stage SM-cycle counters of the fused kernel)
OUT_TRACE = os.path.join(HERE, "_lib_trace")
LIB_TRACE = os.path.join(OUT_TRACE, "libnmc.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    paths += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def build(verbose=False, force=False, debug=False, trace=False):
    """Compile and link libnmc.so (debug: the NMC_DEBUG build; trace: the NMC_TRACE build; each in its
    own folder); returns its path."""
    if debug and trace:
        raise ValueError("the NMC_DEBUG and NMC_TRACE builds are separate")
    out, lib = (OUT_DEBUG, LIB_DEBUG) if debug else ((OUT_TRACE, LIB_TRACE) if trace else (OUT, LIB))
    flags = FLAGS + (["-DNMC_DEBUG"] if debug else []) + (["-DNMC_TRACE"] if trace else [])
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()
    hdr = _headers_mtime()
    jobs = []
    for src in _sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(out, src[:-3] + ".o")
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            jobs.append([nvcc, *flags, *ARCH, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(out, src[:-3] + ".o") for src in _sources()]
    if force or jobs or not os.path.exists(lib):
        run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", lib, *objs])
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, debug="--debug" in sys.argv, trace="--trace" in sys.argv))
