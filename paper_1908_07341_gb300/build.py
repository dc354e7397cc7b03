"""Builds libshaken.so (the C-ABI library of the hot path) in-tree for sm_103a.

The translation units are compiled in parallel with nvcc and linked into
``paper_1908_07341_gb300/libshaken.so``.  No CMake, no network.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libshaken.so")
SOURCES = ["kernels.cu", "api.cu", "noalloc.cu", "batch.cu", "peak.cu", "sampling.cu", "jit.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libshaken.so")
    return exe


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "shaken.h")]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


LIB_DEBUG = os.path.join(PKG, "libshaken_debug.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")


# The device headers that jit.cu compiles at run time, embedded as strings.
JIT_SOURCES = ["device.cuh", "bounds.cuh", "sweep.cuh", "sweep_kernels.cuh", "checkerboard.cuh"]


def _write_jit_sources(build_dir: str) -> None:
    delim = "SHKSRC"
    names, texts = [], []
    for f in JIT_SOURCES:
        with open(os.path.join(CSRC, f)) as fh:
            text = fh.read()
        if ")" + delim + '"' in text:
            raise RuntimeError(f"{f} contains the raw-string delimiter")
        names.append(f'"{f}"')
        texts.append('R"' + delim + "(" + text + ")" + delim + '"')
    out = ("// generated by build.py from " + ", ".join(JIT_SOURCES) + "\n"
           f"static const int kJitSourceCount = {len(JIT_SOURCES)};\n"
           "static const char* const kJitSourceNames[] = {" + ", ".join(names) + "};\n"
           "static const char* const kJitSourceTexts[] = {\n" + ",\n".join(texts) + "\n};\n")
    path = os.path.join(build_dir, "jit_sources.inc")
    old = None
    if os.path.exists(path):
        with open(path) as fh:
            old = fh.read()
    if old != out:
        with open(path, "w") as fh:
            fh.write(out)


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug_bounds: bool = False) -> str:
    """Compile if any source is newer than the library; return the library path.
    debug_bounds builds libshaken_debug.so instead, with every kernel's
    global-memory index checked (-DSHK_DEBUG_BOUNDS, see shk_debug_bounds)."""
    lib_path = LIB_DEBUG if debug_bounds else LIB
    build_dir = BUILD_DEBUG if debug_bounds else BUILD
    if debug_bounds:
        extra_flags = (*extra_flags, "-DSHK_DEBUG_BOUNDS")
    deps = _deps()
    if not force and not _stale(lib_path, deps):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    _write_jit_sources(build_dir)
    extra_flags = (*extra_flags, "-I", build_dir)
    cc = nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
