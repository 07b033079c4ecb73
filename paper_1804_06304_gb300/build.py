"""Build libac.so (the CUDA library behind include/*.h) in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into ``paper_1804_06304_gb300/_build/libac.so``.  ``checked=True`` builds
the bounds-checked variant (``-DAC_CHECKED``: every gather index is tested against
its array and an escape is reported through the status word) into
``_build_checked/libac.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libac.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-Xptxas", "-warn-spills"]


def _sources():
    return sorted(glob.glob(os.path.join(SRC, "*.cu")))


def _deps():
    return sorted(glob.glob(os.path.join(SRC, "*.cu*")) + glob.glob(os.path.join(SRC, "*.h")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def lib_path(checked: bool = False) -> str:
    return os.path.join(OUT + ("_checked" if checked else ""), "libac.so")


def up_to_date(checked: bool = False) -> bool:
    lib = lib_path(checked)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def _compile(src: str, verbose: bool, out: str, extra: list) -> str:
    obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = lib_path(checked)
    if not force and up_to_date(checked):
        return lib
    out = os.path.dirname(lib)
    extra = ["-DAC_CHECKED"] if checked else []
    os.makedirs(out, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, out, extra), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
