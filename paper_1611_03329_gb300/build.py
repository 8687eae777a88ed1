"""Compile the CUDA library (csrc/*.cu) for sm_103a into ``_lib/liblbm_gb300.so``.

The translation units (site kernels, the TMA step kernel, the host C ABI, the allocation-free
residual entry point) are compiled in parallel with nvcc, then linked into one shared library with the CUDA runtime linked statically.  The output stays in the
source tree (``paper_1611_03329_gb300/_lib``, git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB_NAME = "liblbm_gb300.so"
LIB = os.path.join(OUT_DIR, LIB_NAME)
# the bounds-checked variant (-DLBM_BOUNDS_CHECK, see lbm_bounds_report in include/lbm.h)
LIB_CHECKED = os.path.join(OUT_DIR, "liblbm_gb300_checked.so")
SOURCES = ["lbm_kernels.cu", "lbm_tma.cu", "lbm_api.cu", "lbm_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "lbm.h"))
    return files


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(src: str, obj: str, extra: list[str]) -> None:
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build the shared library (or, with checked=True, its bounds-checked variant) if any
    source is newer than it; return its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = (["-Xptxas", "-v"] if verbose else []) + (["-DLBM_BOUNDS_CHECK"] if checked else [])
    tag = "_checked" if checked else ""
    objs = [os.path.join(OUT_DIR, s.replace(".cu", f"{tag}.o")) for s in SOURCES]
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        list(ex.map(lambda a: _compile(a[0], a[1], extra), zip(SOURCES, objs)))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
