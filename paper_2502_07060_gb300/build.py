"""Build of the CUDA library ``libbg.so`` (sm_103a) with nvcc.

Every ``csrc/*.cu`` file is compiled to an object in parallel (one per
field and dimension pair, so the kernel instances spread over all cores),
then linked into ``_build/libbg.so`` with the CUDA runtime linked
statically.  Objects are rebuilt only when their source or a header is
newer.  The multiply-pipe benchmark behind the roofline peaks is built only
on request (``build_pipe_benchmark``).
"""

from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbg.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(obj, src, hdr_mtime):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return t < os.path.getmtime(src) or t < hdr_mtime


def _compile(src, obj, verbose, extra=()):
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr[-4000:]}")
    os.replace(obj + ".tmp", obj)
    return r.stderr


CHECKED_OUT = os.path.join(OUT, "checked")
CHECKED_LIB = os.path.join(CHECKED_OUT, "libbg.so")


def build(jobs=None, verbose=False, force=False, checked=False):
    """Compile and link libbg.so; returns its path.  checked=True builds the
    bounds-checked variant (-DBG_CHECKED) into _build/checked/ instead."""
    out = CHECKED_OUT if checked else OUT
    lib = CHECKED_LIB if checked else LIB
    extra = ["-DBG_CHECKED"] if checked else []
    os.makedirs(os.path.join(out, "obj"), exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_mtime = max(os.path.getmtime(h) for h in _headers())
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(out, "obj", os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, s, hdr_mtime):
            todo.append((s, o))
    # the slowest translation units (the two batch kernels) first, so the
    # pool drains evenly
    def weight(src):
        b = os.path.basename(src)
        return (b.startswith("bg_batch_"), b)
    todo.sort(key=lambda so: weight(so[0]), reverse=True)
    logs = {}
    if todo:
        with ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
            futs = {ex.submit(_compile, s, o, verbose, extra): s for s, o in todo}
            for f, s in futs.items():
                logs[s] = f.result()
    if todo or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, lib)
    if verbose:
        for s, log in logs.items():
            print(f"== {os.path.basename(s)}\n{log}")
    return lib


PEAKS_SRC = os.path.join(CSRC, "peaks", "pipe_throughput.cu")
PEAKS_BIN = os.path.join(OUT, "pipe_throughput")


def build_pipe_benchmark():
    """The stand-alone multiply-pipe benchmark behind the roofline peaks
    (``python -m paper_2502_07060_gb300.build --peaks`` builds it; run it as
    _build/pipe_throughput on a GB300).  Not part of the library build."""
    if os.path.exists(PEAKS_BIN) and os.path.getmtime(PEAKS_BIN) >= os.path.getmtime(PEAKS_SRC):
        return PEAKS_BIN
    tmp = PEAKS_BIN + f".tmp{os.getpid()}"
    subprocess.run([_nvcc(), *ARCH, "-O3", "-o", tmp, PEAKS_SRC], check=True, capture_output=True, text=True)
    os.replace(tmp, PEAKS_BIN)
    return PEAKS_BIN


if __name__ == "__main__":
    import sys
    import time
    t0 = time.time()
    if "--peaks" in sys.argv:
        os.makedirs(OUT, exist_ok=True)
        print(build_pipe_benchmark(), f"{time.time() - t0:.1f}s")
    else:
        print(build(verbose="-v" in sys.argv, force="-f" in sys.argv), f"{time.time() - t0:.1f}s")
