"""Builds the CUDA library libmlswlbm.so in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library with the CUDA runtime linked statically (no dependency on the
runtime PyTorch ships). build(debug=True) makes the bounds-checked variant
libmlswlbm_debug.so (-DMLSW_DEBUG, objects in _lib/debug/), which the tests
build on demand.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libmlswlbm.so")
DEBUG_LIB = os.path.join(OUT_DIR, "libmlswlbm_debug.so")
SOURCES = ["mlswlbm.cu", "step_kernels.cu", "batch_kernels.cu", "aux_kernels.cu", "noalloc.cu",
           "batch.cu", "analysis.cu", "unet.cu"]
HEADERS = ["physics.cuh", "d2q9_tile.cuh", "kernels.h", "tma.cuh", "tcgen05.cuh", "host.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
          "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _deps():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "mlswlbm.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(src, extra, obj_dir=OUT_DIR):
    obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC, *ARCH, *CFLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra=(), debug=False):
    """Compiles the library (the bounds-checked one with debug=True) if a
    source changed; returns its path."""
    lib = DEBUG_LIB if debug else LIB
    if not force and not _stale(lib):
        return lib
    obj_dir = os.path.join(OUT_DIR, "debug") if debug else OUT_DIR
    os.makedirs(obj_dir, exist_ok=True)
    flags = list(extra) + (["-DMLSW_DEBUG"] if debug else [])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, flags, obj_dir), SOURCES))
    if verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    args = sys.argv[1:]
    extra = ["-Xptxas", "-v"] if "--ptxas-v" in args else []
    print(build(force=True, verbose=True, extra=extra))
