"""Builds libwcns.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; the shared library links them with the
static CUDA runtime.  Usage: `python -m paper_2306_09760_gb300.build [--force]`.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwcns.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "--expt-relaxed-constexpr", f"-I{INCLUDE}"]
# Per-unit flags.  Single-precision division, reciprocal and square root use the fast
# approximations (about 2 ulp) and single-precision denormals flush to zero; these flags
# do not touch double precision, so the FP64 path keeps IEEE-rounded operations.
FAST_F32 = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
UNITS = {
    "wcns_api.cu": [],
    "wcns_batch.cu": FAST_F32,
    "wcns_noalloc.cu": [],
    "wcns_f64.cu": [],
    "wcns_f64_x1.cu": [],
    "wcns_f64_x3.cu": [],
    "wcns_f64_x4.cu": [],
    "wcns_f64_y.cu": [],
    "wcns_f64_adj.cu": [],
    "wcns_f64_band.cu": [],
    "wcns_f32.cu": FAST_F32,
    "wcns_f32_x1.cu": FAST_F32,
    "wcns_f32_x3.cu": FAST_F32,
    "wcns_f32_x4.cu": FAST_F32,
    "wcns_f32_y.cu": FAST_F32,
    "wcns_f32_adj.cu": FAST_F32,
    "wcns_f32_band.cu": FAST_F32,
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _sources_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode() + f.read())
    h.update(repr((ARCH, COMMON, UNITS)).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    digest = _sources_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == digest:
        return LIB
    cc = nvcc()

    def compile_one(item):
        src, flags = item
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS.items()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
