"""Build libdq.so (the CUDA library behind include/dq.h) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then the
objects are linked into ``libdq.so`` next to this file.  Rebuilds only when a
source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdq.so")
# The bounds-checking build (DQ_DEBUG_BOUNDS): the same compilation with the
# index checks compiled in (each translation unit keeps its own record of
# failed checks, read by the library).
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libdq_debug.so")
DEBUG_FLAGS = ["-DDQ_DEBUG_BOUNDS"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def cuda_flags():
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
            "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
            f"-I{INCLUDE}", f"-I{CSRC}", f"-I{BUILD}"]


# Device headers the run-time specialised kernels are compiled from (csrc/jit.cu
# hands their texts to NVRTC as in-memory headers).
JIT_HEADERS = [(os.path.join(INCLUDE, "dq.h"), "dq.h")] + [
    (os.path.join(CSRC, h), h) for h in ("dq_common.cuh", "dq_engine.cuh", "dq_tma.cuh", "dq_tile_fwd.cuh",
                                         "dq_tile_adj.cuh", "dq_rows_body.cuh", "dq_devterm.h")]


def write_jit_headers():
    """_build/jit_headers.inc: the device headers as C++ raw strings."""
    os.makedirs(BUILD, exist_ok=True)
    out = ["// generated by build.py from the device headers; do not edit", ""]
    names, texts = [], []
    for path, name in JIT_HEADERS:
        text = open(path).read()
        if ")DQJIT\"" in text:
            raise RuntimeError(f"{name} contains the raw-string delimiter")
        names.append(f'"{name}"')
        texts.append('R"DQJIT(' + text + ')DQJIT"')
    out.append(f"static const int kJitHeaderCount = {len(names)};")
    out.append("static const char *const kJitHeaderNames[] = {" + ", ".join(names) + "};")
    out.append("static const char *const kJitHeaderTexts[] = {")
    out.append(",\n".join(texts))
    out.append("};")
    data = "\n".join(out) + "\n"
    target = os.path.join(BUILD, "jit_headers.inc")
    if not os.path.exists(target) or open(target).read() != data:
        with open(target, "w") as f:
            f.write(data)


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build libdq.so, or with debug=True the bounds-checking libdq_debug.so."""
    lib, bdir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(bdir, exist_ok=True)
    write_jit_headers()
    nvcc = _nvcc()
    extra = DEBUG_FLAGS if debug else []

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *cuda_flags(), *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
