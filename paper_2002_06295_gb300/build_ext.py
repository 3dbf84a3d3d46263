"""Compile the CUDA library libmkf.so for sm_103a (nvcc, in-tree, no torch types).

Each translation unit is compiled in parallel to an object file, then linked.
Objects are rebuilt only when a source or header is newer.
"""
import concurrent.futures as cf
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(HERE, "libmkf.so")
LIB_ARCH = LIB + ".arch"   # machine the library was linked for
SOURCES = ["abi.cu", "bin_hits.cu", "build.cu", "dedup.cu", "fit.cu", "fit_adjoint.cu", "overlaps.cu", "seeds.cu", "strips.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "--expt-relaxed-constexpr"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps():
    out = [os.path.join(INCLUDE, "mkf.h")]
    for f in os.listdir(CSRC):
        if f.endswith((".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    srcp = os.path.join(CSRC, src)
    newest = max(os.path.getmtime(p) for p in [srcp] + _deps())
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest and not verbose_ptxas:
        return obj, ""
    cmd = [_nvcc()] + ARCH + FLAGS + (["-Xptxas", "-v"] if verbose_ptxas else []) + ["-c", srcp, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(verbose_ptxas=False, quiet=True):
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    objs = [o for o, _ in res]
    if verbose_ptxas:
        for (o, log), s in zip(res, SOURCES):
            print("==", s)
            print(log)
    newest = max(os.path.getmtime(o) for o in objs)
    arch_ok = os.path.exists(LIB_ARCH) and open(LIB_ARCH).read().strip() == platform.machine()
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest or not arch_ok:
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
        with open(LIB_ARCH, "w") as f:
            f.write(platform.machine())
    if not quiet:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose_ptxas="-v" in sys.argv, quiet=False)
