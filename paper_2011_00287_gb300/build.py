"""Builds liblbcad.so in-tree with nvcc for sm_103a (translation units compiled in
parallel, no cmake).  Output: paper_2011_00287_gb300/_lib/liblbcad.so."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblbcad.so")
# arithmetic-throughput probes for the bench's roofline denominators (not part of the step)
PEAKS_LIB = os.path.join(LIBDIR, "libpeaks.so")
UNITS = ["lbcad_runtime.cu", "lbcad_f32.cu", "lbcad_f64.cu", "lbcad_noalloc.cu", "lbcad_adj_f32.cu",
         "lbcad_adj_f64.cu"]
# Units with FP32 kernels flush FP32 subnormals to zero.  Subnormal values (below 1.2e-38)
# appear where the first disturbances spread into the quiescent fluid around the droplet and
# slow the FP32 arithmetic: the 128^3 step took 0.306 ms over its first 50 steps and 0.240
# ms later, against 0.234 ms throughout when flushed.  They lie some 30 orders of magnitude
# below the FP32 resolution of every field.  (-ftz leaves FP64 arithmetic alone.)
FTZ_UNITS = {"lbcad_f32.cu", "lbcad_noalloc.cu", "lbcad_adj_f32.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + [
        os.path.join(ROOT, "include", "lbcad.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PEAKS_LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    flags = ["-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xptxas", "-v",
             "-Xcompiler", "-fPIC,-ffp-contract=off", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]

    def compile_one(u):
        src = os.path.join(CSRC, u)
        obj = os.path.join(OBJ, u.replace(".cu", ".o"))
        extra = ["-ftz=true"] if u in FTZ_UNITS else []
        r = subprocess.run([cc, *flags, *extra, "-c", src, "-o", obj], capture_output=True, text=True)
        with open(obj + ".log", "w") as fh:
            fh.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (u, r.stderr[-4000:]))
        return obj

    with cf.ThreadPoolExecutor(len(UNITS) + 1) as ex:
        objs = list(ex.map(compile_one, UNITS + ["peaks.cu"]))
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.run([cc, "-shared", *ARCH, "-o", tmp, *objs[:-1]], check=True)
    os.replace(tmp, LIB)
    tmp = PEAKS_LIB + ".%d.tmp" % os.getpid()
    subprocess.run([cc, "-shared", *ARCH, "-o", tmp, objs[-1]], check=True)
    os.replace(tmp, PEAKS_LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
