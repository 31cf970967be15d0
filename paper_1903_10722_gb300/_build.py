"""Build the CUDA library libffs_gb300.so in-tree with nvcc for sm_103a.

Each .cu file is compiled in its own nvcc process (in parallel) and the
objects are linked into one shared library with the CUDA runtime linked
statically.  Output: paper_1903_10722_gb300/_build/libffs_gb300.so, and the
variant with device-side checks (-DFFS_DEBUG_CHECKS: index bounds at the GA's
indexing sites and permutation validity of every generation's rows, recorded
in a device error word) in _build_debug/libffs_gb300_debug.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libffs_gb300.so")
OUT_DIR_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DIR_DEBUG, "libffs_gb300_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# relocatable device code: the decoder's per-round functions are compiled once
# (ffs_decoder_*.cu) and called from the kernels of the other units
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-rdc=true"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps() -> list[str]:
    d = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    d.append(os.path.join(os.path.dirname(HERE), "include", "ffs.h"))
    return d


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build_all(force: bool = False) -> list[str]:
    """The library and its checked variant."""
    return [build(force=force), build(force=force, debug=True)]


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, debug: bool = False) -> str:
    out_dir, lib = (OUT_DIR_DEBUG, LIB_DEBUG) if debug else (OUT_DIR, LIB)
    if not force and up_to_date(debug):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    if debug:
        extra = [*(extra or []), "-DFFS_DEBUG_CHECKS"]
    # the decoder units are the longest compiles: start them first
    srcs = sorted(sources(), key=lambda p: (0 if "ffs_decoder" in p else 1, p))
    objs = [os.path.join(out_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(pair):
        src, obj = pair
        # the per-round functions run inside kernels launched with up to 512
        # threads: at most 128 registers (the kernels' launch bounds)
        regs = ["-maxrregcount=128"] if "ffs_decoder" in os.path.basename(src) else []
        cmd = [nvcc, *ARCH, *FLAGS, *regs, *(extra or []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        list(ex.map(compile_one, zip(srcs, objs)))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-rdc=true", "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
