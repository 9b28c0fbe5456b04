"""Build libgrlb.so (CUDA, sm_103a) in-tree with nvcc.

    python -m paper_2609_16361_b300.build [--verbose] [--checked]

The library lands next to this file so it travels with the source tree.  --checked builds
libgrlb_checked.so instead: the same sources compiled with GRLB_CHECKED (every kernel access
tested against the registry of live device regions) and relocatable device code, so that the
kernels of every source file share the one registry.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgrlb.so")
LIB_CHECKED = os.path.join(HERE, "libgrlb_checked.so")
SOURCES = ["grlb_kernels.cu", "grlb_spectral.cu", "grlb_init_ce.cu", "grlb_halo.cu", "grlb_cells.cu", "grlb_check.cu",
           "grlb_api.cu"]
HEADERS = ["grlb_device.cuh", "grlb_kernels.h", "grlb_check.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The sweep, initialisation and probe kernels' arithmetic is fixed by the source: no multiply-add
# contraction by the compiler (every fused multiply-add is an explicit fmaf / fma), so the
# rounding of each operation is the same in every kernel a device function is instantiated in,
# whatever its launch bounds, register budget or surrounding code -- the condition for moment
# and population storage, the checked build, the batched and the diagnostic sweeps to agree bit
# for bit.  The spectral file keeps the compiler's contraction: its fusions written out ran
# 1.48 against 1.44 ms per 256^3 call, and no two of its kernels need to agree bit for bit.
FILE_FLAGS = {f: ["-fmad=false"] for f in ("grlb_kernels.cu", "grlb_init_ce.cu", "grlb_cells.cu")}


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def needs_build(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "grlb.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every source file to an object in parallel, then link the shared library."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not needs_build(checked):
        return lib
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
             "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if checked:
        flags += ["-DGRLB_CHECKED", "-rdc=true"]
    if verbose:
        flags += ["-Xptxas", "-v"]
    with tempfile.TemporaryDirectory(prefix="grlb_build_") as tmpdir:
        objs = [os.path.join(tmpdir, f[:-3] + ".o") for f in SOURCES]
        jobs = [[_nvcc(), *flags, *FILE_FLAGS.get(f, []), "-c", os.path.join(CSRC, f), "-o", o]
                for f, o in zip(SOURCES, objs)]
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
            for rc, cmd in zip(ex.map(subprocess.call, jobs), jobs):
                if rc != 0:
                    raise subprocess.CalledProcessError(rc, cmd)
        tmp = lib + f".tmp{os.getpid()}"
        link = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        if checked:
            link.insert(1, "-rdc=true")  # device link: the kernels of all files share one registry
        subprocess.check_call(link)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="--verbose" in sys.argv, checked="--checked" in sys.argv))
