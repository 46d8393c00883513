"""Build libqrs.so in-tree: every CUDA translation unit compiled for sm_103a
in parallel with nvcc, then linked into one shared library next to this file.

Usage: python -m paper_2404_02978_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libqrs.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills",
         "--expt-relaxed-constexpr"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(HERE, "..", "include", "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), out: str = None, build_dir: str = None) -> str:
    """Compile and link libqrs.so.  `extra` adds nvcc flags (e.g. -D tunables);
    `out` / `build_dir` place a variant build elsewhere (then it always rebuilds)."""
    OUT_ = out or OUT
    BUILD_ = build_dir or BUILD
    if not force and out is None and up_to_date():
        return OUT
    os.makedirs(BUILD_, exist_ok=True)
    nvcc = _nvcc()
    srcs = sources()

    def one(src):
        obj = os.path.join(BUILD_, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-I", CSRC, "-I", os.path.join(HERE, "..", "include"),
               "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(one, srcs))
    tmp = OUT_ + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lcudart", "-lcuda"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, OUT_)
    return OUT_


CHECKED_OUT = os.path.join(HERE, "libqrs_checked.so")


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The bounds-checked library (QRS_CHECKED=1, libqrs_checked.so): every
    checked accessor in the kernels tests its index against its buffer's
    extent (include/qrs.h, "bounds-checked build").  Loaded by the binding
    instead of libqrs.so when QRS_CHECKED=1 is set in the environment."""
    if not force and os.path.exists(CHECKED_OUT) and all(
            os.path.getmtime(d) <= os.path.getmtime(CHECKED_OUT) for d in _deps()):
        return CHECKED_OUT
    return build(verbose=verbose, extra=["-DQRS_CHECKED=1"], out=CHECKED_OUT,
                 build_dir=os.path.join(HERE, "_build_checked"))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
