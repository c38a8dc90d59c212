"""Compile the CUDA library libmehdg.so in-tree for sm_103a (nvcc, no cmake)."""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmehdg.so")
LIB_BOUNDS_CHECK = os.path.join(HERE, "libmehdg_bc.so")
SOURCES = ["reference.cpp", "condense.cu", "apply.cu", "apply_fix.cu", "krylov.cu", "krylov_fix.cu", "api.cu", "static_scratch.cu", "adjoint.cu", "apply_mrhs.cu", "levels.cu", "precond.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _compile(src, extra, build_dir=BUILD):
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj, res.stderr


def build(verbose=False, extra=(), lib=LIB, build_dir=BUILD):
    """Compile every translation unit in parallel and link libmehdg.so (or `lib`, e.g. the
    bounds-checked variant: extra=("-DHDG_BOUNDS_CHECK",), lib=LIB_BOUNDS_CHECK)."""
    os.makedirs(build_dir, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra), build_dir), SOURCES))
    objs = [r[0] for r in results]
    if verbose:
        for _, log in results:
            if log:
                print(log)
    tmp = lib + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


def build_bounds_checked(verbose=False):
    """The bounds-checked variant of the library (every guarded device index checked, the
    first failure recorded and the access skipped), in-tree beside the regular one."""
    return build(verbose, extra=("-DHDG_BOUNDS_CHECK",), lib=LIB_BOUNDS_CHECK,
                 build_dir=os.path.join(HERE, "_build_bc"))


if __name__ == "__main__":
    print(build(verbose=True))
