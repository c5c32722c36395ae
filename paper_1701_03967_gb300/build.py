"""Build libfemfft.so in-tree with nvcc for sm_103a (no torch extension
machinery: the library has a plain C ABI).  The translation units are
compiled in parallel, then linked."""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfemfft.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["pencil_f64.cu", "pencil_f32.cu", "pencil_fast_f32_v16.cu", "pencil_fast_f32_v32.cu", "apply.cu",
              "api.cu", "noalloc.cu", "batch.cu", "batch_k1.cu", "batch_k2.cu", "batch_k3.cu", "band.cu",
              "dirichlet.cu", "host.cu", "longpass.cu"]
CPP_SOURCES = ["precompute.cpp", "pencil_fast_plan.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose=False, force=False):
    """Compile every translation unit and link libfemfft.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    srcs = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES]
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "femfft.h"))
    newest_dep = max(os.path.getmtime(f) for f in srcs + headers)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest_dep:
        return LIB
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(os.path.dirname(HERE), "include")]
    newest_header = max(os.path.getmtime(f) for f in headers)
    jobs = []
    objs = []

    def stale(src, obj):
        # an object is rebuilt when its source or any header is newer
        return force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), newest_header)

    for f in CU_SOURCES:
        src, obj = os.path.join(CSRC, f), os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if stale(src, obj):
            jobs.append([nvcc] + ARCH + common + ["-lineinfo", "-Xptxas", "-v", "-c", src, "-o", obj])
    for f in CPP_SOURCES:
        src, obj = os.path.join(CSRC, f), os.path.join(BUILD, f + ".o")
        objs.append(obj)
        # the double-double precompute needs IEEE operations without contraction
        if stale(src, obj):
            jobs.append([nvcc] + common + ["-Xcompiler", "-ffp-contract=off", "-c", src, "-o", obj])
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIB + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
