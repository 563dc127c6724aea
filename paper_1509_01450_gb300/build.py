"""Build libsgdisk.so (the CUDA path for sm_103a) in place.

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into paper_1509_01450_gb300/libsgdisk.so.  Usage:

    python -m paper_1509_01450_gb300.build [--force] [--verbose-ptxas] [--checked]

--checked builds the index-checked variant instead (-DSG_DEBUG, objects in
_build_checked/, paper_1509_01450_gb300/libsgdisk_checked.so; loaded when
SG_LIBRARY_VARIANT=checked).  Extra nvcc options may come from the
environment variable SG_NVCC_FLAGS (split on white space); the objects are
rebuilt whenever they change.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsgdisk.so")
OBJ_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libsgdisk_checked.so")
# fftconv_lg<LG>.cu compile the fixed-length instances of fftconv.cu's pass
# kernels, one transform length each, in parallel with the rest
SOURCES = ["api.cu", "batch.cu", "dft_tc.cu", "kbuild.cu", "fftconv.cu", "fftconv_df.cu", "noalloc.cu", "wedge.cu"] + [f"fftconv_lg{lg}.cu" for lg in range(8, 14)]
HEADERS = ["sg_common.cuh", "sg_df.cuh", "sg_internal.cuh", "sg_tc.cuh", "fftconv.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = False) -> str:
    obj_dir, lib_path = (OBJ_CHECKED, LIB_CHECKED) if checked else (OBJ, LIB)
    os.makedirs(obj_dir, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "sg.h")]
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
    extra = os.environ.get("SG_NVCC_FLAGS", "").split() + (["-DSG_DEBUG"] if checked else [])
    flags += extra
    # a change of the extra options rebuilds every object
    stamp = os.path.join(obj_dir, "flags.txt")
    old = open(stamp).read() if os.path.exists(stamp) else None
    if old != " ".join(extra):
        force = True
        with open(stamp, "w") as f:
            f.write(" ".join(extra))
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(obj_dir, src.replace(".cu", ".o"))
        if force or verbose_ptxas or _stale(o, [s] + hdrs):
            jobs.append([nvcc()] + flags + ["-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            procs = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, p in zip(jobs, procs):
            if p.returncode != 0 or verbose_ptxas:
                sys.stderr.write(p.stdout + p.stderr)
            if p.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    objs = [os.path.join(obj_dir, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + ".tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            sys.stderr.write(p.stdout + p.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--verbose-ptxas" in sys.argv,
                checked="--checked" in sys.argv))
