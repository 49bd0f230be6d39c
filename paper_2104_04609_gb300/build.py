"""In-tree build of the CUDA library libosrc_pmchwt.so for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2104_04609_gb300/_build/libosrc_pmchwt.so.  No CMake, one -gencode."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libosrc_pmchwt.so")
SOURCES = ["osrc_api.cu", "k_far.cu", "k_near.cu", "k_sparse.cu", "k_gmres.cu", "k_rhs.cu",
           "server.cu", "k_dense.cu", "k_batched.cu", "k_field.cu", "k_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
# per-file flags: the FP32 far-field kernel flushes FP32 subnormals (its
# values are far from the subnormal range), which removes subnormal handling
# around the MUFU reciprocal square root and sine / cosine
FILE_FLAGS = {"k_far.cu": ["-ftz=true"]}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.abspath(__file__), os.path.join(CSRC, "osrc_internal.cuh"), os.path.join(CSRC, "ffmath.cuh"),
              os.path.join(CSRC, "stream_k.cuh"), os.path.join(CSRC, "dense_sched.cuh"),
              os.path.join(os.path.dirname(HERE), "include", "osrc_pmchwt.h")]
    return files


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB):
        lib_m = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) <= lib_m for f in _deps()):
            return LIB
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *FILE_FLAGS.get(src, []), *extra, "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    extra = [a for a in sys.argv[1:] if a.startswith("-X")]
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, extra=extra))
