"""Builds libsecpe.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a) and the objects are linked into
paper_2502_00847_gb300/_build/libsecpe.so.  No cmake, no torch extension.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libsecpe.so")

SOURCES = ["hostmath.cpp", "context.cu", "ntt.cu", "ntt_fused.cu", "kernels.cu", "keyswitch.cu", "eval.cu",
           "capi.cu", "encode.cpp", "noalloc.cu", "server.cu", "ntt_tc.cu", "linear.cu", "boot.cu", "ntt32.cu"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-I" + os.path.join(ROOT, "include")]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src):
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(
            os.path.getmtime(path),
            *[os.path.getmtime(os.path.join(CSRC, h)) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))],
            os.path.getmtime(os.path.join(ROOT, "include", "secpe.h"))):
        return obj
    cmd = [nvcc(), "-c", path, "-o", obj] + COMMON
    if src.endswith(".cu"):
        cmd += ARCH + ["-lineinfo", "--expt-relaxed-constexpr"]
    else:
        cmd += ["-x", "c++"]
    subprocess.check_call(cmd)
    return obj


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    if os.path.exists(SO) and os.path.getmtime(SO) >= max(os.path.getmtime(o) for o in objs):
        return SO
    tmp = SO + ".tmp%d" % os.getpid()
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "-lcudart_static"]
    subprocess.check_call(cmd)
    os.replace(tmp, SO)
    if verbose:
        print("built", SO)
    return SO


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
