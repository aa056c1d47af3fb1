"""Builds libmdgb.so (the CUDA hot path behind include/md.h) in-tree.

Each .cu translation unit is compiled for sm_103a in parallel, then linked
into one shared library with the shared CUDA runtime.  Output:
paper_1412_3387_gb300/_build/libmdgb.so (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmdgb.so")
RATE_LIB = os.path.join(BUILD, "libmdrate.so")  # FP64 rate microbenchmark (not the MD ABI)
SOURCES = ["api.cu", "k_cells.cu", "k_nlist.cu", "k_pair.cu", "k_pair_lj_mixed.cu",
           "k_pair_lj_fp64.cu", "k_pair_dpd_mixed.cu", "k_pair_dpd_fp64.cu",
           "k_pair_gauss_mixed.cu", "k_pair_gauss_fp64.cu", "k_pair_morse_mixed.cu",
           "k_pair_morse_fp64.cu", "k_pair_yukawa_mixed.cu", "k_pair_yukawa_fp64.cu",
           "k_pair_table_mixed.cu", "k_pair_table_fp64.cu",
           "k_integrate.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-D__NV_NO_VECTOR_DEPRECATION_DIAG", *extra]


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, "md_internal.cuh"), os.path.join(CSRC, "brick.cuh"),
               os.path.join(CSRC, "pair_impl.cuh"),
               os.path.join(ROOT, "include", "md.h"),
               os.path.abspath(__file__)]
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or ptxas_info or _stale(o, [s] + headers):
            cmd = [cc, *_flags(extra), "-c", s, "-o", o + ".tmp"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
            if verbose or ptxas_info:
                sys.stderr.write(r.stderr)
            os.replace(o + ".tmp", o)
        return o

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        objs = list(ex.map(compile_one, SOURCES + ["fp64_rate.cu"]))
    rate_obj = objs.pop()
    if force or _stale(RATE_LIB, [rate_obj]):
        tmp = RATE_LIB + f".{os.getpid()}.tmp"
        r = subprocess.run([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, rate_obj,
                            "-Xlinker", "-rpath,/usr/local/cuda/lib64"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, RATE_LIB)
    if force or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
