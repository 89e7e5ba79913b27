"""Build the CUDA library libbiharm.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into a
shared library next to this file.  Used by ``__graft_entry__.build()`` and by
``python -m paper_2412_05082_gb300.build``.
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
LIB = os.path.join(HERE, "libbiharm.so")
# the longest translation units first
SOURCES = ["defect_ff_k7.cu", "defect_ff_k6.cu", "batch_pers_f64.cu", "batch_pers_f32.cu",
           "defect_ff_k5.cu", "defect_ff_k2_4.cu", "inst_f64.cu", "inst_f32.cu",
           "batch_mvs_f64.cu", "batch_mvs_f32.cu", "batch.cu", "vec.cu", "api.cu", "setup.cpp",
           "noalloc.cu", "serve.cpp", "probe.cu", "gemm.cu", "defect_ff.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        exe = "/usr/local/cuda/bin/nvcc"
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbiharm.so")
    return exe


def _compile(src, extra=()):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp",
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, *extra,
           "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "cu")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), res.stderr))
    return obj


def build(verbose=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), res.stderr))
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
