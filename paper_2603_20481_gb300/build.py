"""Build the RISE CUDA library (librise.so) in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked into
paper_2603_20481_gb300/_lib/librise.so with a static CUDA runtime.

`--checked` builds the checked variant instead (-DRISE_CHECKED, into
_lib_checked/librise_checked.so): every data-dependent index is checked on
the device, a failed check is reported as RISE_EINTERNAL, and nothing is
accessed out of range.  The binding loads it when RISE_CHECKED=1 is set.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "librise.so")
CHECKED_DIR = os.path.join(HERE, "_lib_checked")
CHECKED_LIB = os.path.join(CHECKED_DIR, "librise_checked.so")
SOURCES = ["stft.cu", "stft_s1.cu", "stft_s2.cu", "stft_sc16.cu", "image.cu", "ccl.cu", "rise.cu", "batch.cu",
           "server.cu", "match.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "common.cuh"), os.path.join(CSRC, "context.cuh"),
            os.path.join(CSRC, "stft_impl.cuh"),
            os.path.join(os.path.dirname(HERE), "include", "rise.h")]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    out_dir, lib = (CHECKED_DIR, CHECKED_LIB) if checked else (OUT_DIR, LIB)
    if checked:
        extra = (*extra, "-DRISE_CHECKED")
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        if force or _stale(o, s):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {cmd[-3]}")
        return r

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(out_dir, s.replace(".cu", ".o")) for s in SOURCES]
    if jobs or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    extra = ["-Xptxas", "-v"] if "-v" in sys.argv else []
    print(build(force="--force" in sys.argv, verbose=bool(extra), extra=extra,
                checked="--checked" in sys.argv))
