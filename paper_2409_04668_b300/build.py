"""Builds the CUDA library ``libmcdc_b300.so`` in-tree for sm_103a, and its
checked twin ``libmcdc_b300_checks.so`` (compiled with ``-DMCDC_CHECKS``:
every kernel index bounds-checked before its access).

Every kernel is compiled with ``-gencode arch=compute_103a,code=sm_103a``.
The FP64 tracker and the reduction kernels are compiled with ``-fmad=false``
so that their arithmetic is rounded operation by operation, as written.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmcdc_b300.so")
BUILD_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(HERE, "libmcdc_b300_checks.so")

NVCC = os.environ.get("NVCC", shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
NO_FMA = {"track_fp64.cu", "misc.cu", "comb.cu"}


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    out.append(os.path.join(ROOT, "include", "mcdc.h"))
    return out


def _compile(src, extra, bdir=BUILD):
    obj = os.path.join(bdir, src.replace(".cu", ".o"))
    flags = list(COMMON) + (["-fmad=false"] if src in NO_FMA else []) + list(extra)
    cmd = [NVCC] + ARCH + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r.returncode, r.stdout + r.stderr


def build(force=False, verbose=False, extra=(), checked=False):
    """Builds the library (checked: the bounds-checked twin) unless it is
    newer than every source; returns its path."""
    bdir, lib = (BUILD_CHECKS, LIB_CHECKS) if checked else (BUILD, LIB)
    extra = list(extra) + (["-DMCDC_CHECKS"] if checked else [])
    os.makedirs(bdir, exist_ok=True)
    srcs = sources()
    deps = [os.path.join(CSRC, s) for s in srcs] + headers() + [os.path.abspath(__file__)]
    if not force and os.path.exists(lib):
        m = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= m for d in deps):
            return lib
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, bdir), srcs))
    ok = True
    for src, obj, rc, log in results:
        if rc != 0 or verbose:
            sys.stderr.write(f"--- {src} (rc={rc})\n{log}\n")
        ok = ok and rc == 0
    if not ok:
        raise RuntimeError("nvcc failed")
    tmp = lib + f".tmp{os.getpid()}"
    objs = [o for _, o, _, _ in results]
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


def build_all(force=False):
    """The library and its checked twin."""
    return build(force=force), build(force=force, checked=True)


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(extra), extra=extra))
    if "--no-checks" not in sys.argv:
        print(build(force=True, verbose=v, checked=True))
