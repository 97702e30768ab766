"""Build the CUDA library in-tree: paper_2602_14493_b300/libgmr.so.

nvcc for sm_103a only (-gencode arch=compute_103a,code=sm_103a), -O3,
-lineinfo, static CUDA runtime, one shared object exporting the C ABI of
include/gmr.h (the sources compiled in parallel, then linked). Cross-compiles
without a GPU.
"""

from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgmr.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "gmr.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
             "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags += ["-Xptxas", "-v"]
    # one nvcc per source file, in parallel, then one link
    objdir = tempfile.mkdtemp(prefix="gmr_build_")
    try:
        objs = [os.path.join(objdir, os.path.basename(src) + ".o") for src in sources()]
        with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
            for r in ex.map(lambda so: subprocess.run([NVCC, *flags, "-c", so[0], "-o", so[1]]),
                            zip(sources(), objs)):
                if r.returncode != 0:
                    raise subprocess.CalledProcessError(r.returncode, r.args)
        subprocess.run([NVCC, *ARCH, "-shared", "-cudart", "static", "-o", LIB + ".tmp", *objs], check=True)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
