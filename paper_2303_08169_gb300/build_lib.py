"""Build the in-tree shared library libpaper_2303_08169_gb300.so for sm_103a.

Steps: compile and run the tensor-product code generator (g++), compile every
CUDA translation unit with nvcc in parallel, link one shared library next to
this file.  Build products other than the .so live in <repo>/_build.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIBNAME = "libpaper_2303_08169_gb300.so"
LIB = os.path.join(HERE, LIBNAME)
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["neighbor.cu", "model_fp32.cu", "model_fp32_o3.cu", "model_bf16.cu", "md.cu", "api.cu", "umma_selftest.cu", "noalloc.cu", "train.cu"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}")
    if verbose and r.stdout.strip():
        print(r.stdout)
    return r.stdout


def build(verbose=False, extra_flags=()):
    os.makedirs(BUILD, exist_ok=True)
    gen = os.path.join(BUILD, "gen_tp")
    _run(["g++", "-O2", "-std=c++17", "-o", gen, os.path.join(CSRC, "gen_tp.cpp")], verbose)
    _run([gen, os.path.join(BUILD, "tp_tables.inc")], verbose)
    nvcc = _nvcc()
    flags = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
             "--expt-relaxed-constexpr", "-I", BUILD, "-I", os.path.join(ROOT, "include"),
             *extra_flags]
    objs = []
    jobs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        for src in SOURCES:
            obj = os.path.join(BUILD, src.replace(".cu", ".o"))
            objs.append(obj)
            jobs.append(ex.submit(_run, [nvcc, *flags, "-c", os.path.join(CSRC, src), "-o", obj], verbose))
        for j in jobs:
            j.result()
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", ARCH, "-o", tmp, *objs], verbose)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
