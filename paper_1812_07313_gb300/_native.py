"""Build and load the package's native libraries (in-tree, under ``_build/``).

  * ``libqg_tree.so`` -- host oct-tree / group walk (g++, OpenMP)
  * ``libqgrav.so``   -- the CUDA hot path behind the ``qg_*`` C-ABI
                         (nvcc, sm_103a only)

Both are rebuilt when a source or header is newer than the library.  Nothing
here falls back to Python: if a library cannot be built or loaded the caller
gets the compiler's or loader's error.
"""
from __future__ import annotations

import ctypes
import glob
import os
import shutil
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")

TREE_LIB = os.path.join(BUILD, "libqg_tree.so")
CUDA_LIB = os.path.join(BUILD, "libqgrav.so")

CUDA_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Per-source extra flags: the FP32 force kernels flush single-precision
# denormals (one SFU instruction per reciprocal square root, no fix-up path).
CUDA_FLAGS = {"qg_force_f32.cu": ["-ftz=true"], "qg_force_f32x2.cu": ["-ftz=true"],
              "qg_force_f32ep.cu": ["-ftz=true"], "qg_noalloc.cu": ["-ftz=true"],
              "qg_force_adapt.cu": ["-ftz=true"], "qg_force_inplace_adapt.cu": ["-ftz=true"],
              "qg_force_inplace.cu": ["-ftz=true"],
              # the GPU tree reproduces the host builder bit for bit: no FMA
              # contraction on either side
              "qg_gtree.cu": ["-fmad=false", "-Xcompiler", "-ffp-contract=off"]}

_lock = threading.Lock()


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA hot path cannot be built")


def build_tree(force=False, verbose=False):
    srcs = [os.path.join(CSRC, "qg_tree.cpp")]
    deps = srcs + [os.path.join(INCLUDE, "qg_tree.h")]
    with _lock:
        if force or _newer(TREE_LIB, deps):
            os.makedirs(BUILD, exist_ok=True)
            tmp = TREE_LIB + ".tmp%d" % os.getpid()
            cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                   "-I" + INCLUDE] + srcs + ["-o", tmp]
            if verbose:
                print(" ".join(cmd))
            subprocess.check_call(cmd)
            os.replace(tmp, TREE_LIB)
    return TREE_LIB


def cuda_sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def build_cuda(force=False, verbose=False, extra_flags=()):
    """Compile every .cu under csrc/ for sm_103a into one shared library."""
    srcs = cuda_sources()
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    with _lock:
        if force or _newer(CUDA_LIB, deps):
            os.makedirs(BUILD, exist_ok=True)
            nvcc = _nvcc()
            objs = []
            procs = []
            for s in srcs:
                o = os.path.join(BUILD, os.path.basename(s) + ".o")
                objs.append(o)
                cmd = [nvcc] + CUDA_ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                            "-I" + INCLUDE, "-I" + CSRC, "-c", s, "-o", o] + list(extra_flags) \
                    + CUDA_FLAGS.get(os.path.basename(s), [])
                if verbose:
                    print(" ".join(cmd))
                procs.append((cmd, subprocess.Popen(cmd)))
            for cmd, p in procs:
                if p.wait() != 0:
                    raise RuntimeError("nvcc failed: " + " ".join(cmd))
            tmp = CUDA_LIB + ".tmp%d" % os.getpid()
            cmd = [nvcc] + CUDA_ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lcuda"]
            if verbose:
                print(" ".join(cmd))
            subprocess.check_call(cmd)
            os.replace(tmp, CUDA_LIB)
    return CUDA_LIB


def load(path):
    return ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
