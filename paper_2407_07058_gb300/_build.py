"""Builds libappd.so in-tree with nvcc for sm_103a (no torch extension machinery)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libappd.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["appd_api.cu", "mst_kernels.cu", "leaf_order.cu", "fill.cu", "server.cu", "batched.cu",
           "noalloc.cu", "tune.cu", "insert.cu", "contract_tma.cu", "points.cu",
           "insert_tree.cu"]
HEADERS = ["common.cuh", "internal.h", "mst_device.cuh", "leaf_device.cuh", "fill_device.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]

_LOCK = threading.Lock()


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "appd.h"))
    return [f for f in files if os.path.exists(f)]


def lib_path() -> str:
    return LIB


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
    cmd = ["nvcc", *ARCH, *FLAGS, *extra, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile every .cu of the library in parallel and link libappd.so."""
    with _LOCK:
        if not force and not is_stale():
            return LIB
        os.makedirs(OUT_DIR, exist_ok=True)
        srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
        with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
            objs = list(ex.map(lambda s: _compile(s, extra or []), srcs))
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        if verbose:
            print(f"built {LIB}")
        return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
