"""Seeded synthetic inputs shaped like the paper's workloads.

Input generation only: nothing in this package computes minimax distances.
The CUDA library's tests and benchmark, and the CPU oracle, all take their
weight matrices from here, so both sides see the same bytes.

The paper measures on seven point datasets that are not available here
(Section 4.1, Table 2); these generators stand in for them with dense
complete graphs built from seeded point clouds (Gaussian mixtures, uniform
points) and seeded hashed integer weights.

Host matrices come from ``synth.c`` (FP64 distance arithmetic, no FMA,
correctly rounded sqrt, rounded to FP32); large matrices can be produced on
the device by ``synth_cuda.cu`` with the same arithmetic (see
``device_euclid``), which is checked against the host on sampled rows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB = None
_CUDA_LIB = None


def build_host() -> str:
    """Compile synth.c into a shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libsynth.so")
    src = os.path.join(_HERE, "synth.c")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", "-pthread", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def build_cuda() -> str:
    """Compile synth_cuda.cu (device twin of the generators) for sm_103a."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libsynth_cuda.so")
    src = os.path.join(_HERE, "synth_cuda.cu")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "-shared",
                               "-o", tmp, src])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build_host())
            lib.synth_mix64.restype = ctypes.c_uint64
            lib.synth_mix64.argtypes = [ctypes.c_uint64]
            lib.synth_hash.restype = ctypes.c_uint64
            lib.synth_hash.argtypes = [ctypes.c_uint64] * 3
            lib.synth_euclid_f32.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_int]
            lib.synth_hash_u32.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_int]
            lib.synth_uniform01_f32.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_int]
            lib.synth_euclid_row.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                             ctypes.c_int64, ctypes.c_void_p]
            lib.synth_euclid32_f32.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_int]
            _LIB = lib
    return _LIB


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


# ----------------------------------------------------------------- points
def gmm_points(n: int, d: int, k: int, *, sigma: float, seed: int,
               mean_box: float | None = None, mean_std: float | None = None) -> np.ndarray:
    """Equal-weight Gaussian mixture in d dimensions, FP32 coordinates.

    Means are uniform in [0, mean_box]^d or normal with std ``mean_std``.
    """
    rng = np.random.default_rng(seed)
    if mean_box is not None:
        means = rng.random((k, d)) * mean_box
    else:
        means = rng.standard_normal((k, d)) * float(mean_std)
    lab = rng.integers(0, k, size=n)
    pts = means[lab] + sigma * rng.standard_normal((n, d))
    return np.ascontiguousarray(pts.astype(np.float32))


def uniform_points(n: int, d: int, *, seed: int, box: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray((rng.random((n, d)) * box).astype(np.float32))


# --------------------------------------------------------------- matrices
def euclid(points: np.ndarray) -> np.ndarray:
    """FP32 Euclidean distance matrix of FP32 points (definition in synth.c)."""
    pts = np.ascontiguousarray(points, dtype=np.float32)
    n, d = pts.shape
    W = np.empty((n, n), dtype=np.float32)
    if _lib().synth_euclid_f32(pts.ctypes.data, n, d, W.ctypes.data, _threads()) != 0:
        raise RuntimeError("synth_euclid_f32 failed")
    return W


def euclid32(points: np.ndarray) -> np.ndarray:
    """FP32 Euclidean matrix computed in FP32 arithmetic: s = fma(t, t, s) over
    the coordinates in order with t = x_lo,k - x_hi,k, then a correctly rounded
    sqrt (the serving mix's point requests; definition in synth.c)."""
    pts = np.ascontiguousarray(points, dtype=np.float32)
    n, d = pts.shape
    W = np.empty((n, n), dtype=np.float32)
    if _lib().synth_euclid32_f32(pts.ctypes.data, n, d, W.ctypes.data, _threads()) != 0:
        raise RuntimeError("synth_euclid32_f32 failed")
    return W


def euclid_row(points: np.ndarray, i: int) -> np.ndarray:
    pts = np.ascontiguousarray(points, dtype=np.float32)
    n, d = pts.shape
    row = np.empty(n, dtype=np.float32)
    _lib().synth_euclid_row(pts.ctypes.data, n, d, int(i), row.ctypes.data)
    return row


def hash_u32(n: int, seed: int) -> np.ndarray:
    """Symmetric uint32 weights uniform in [0, 2^16), zero diagonal."""
    W = np.empty((n, n), dtype=np.uint32)
    _lib().synth_hash_u32(seed, n, W.ctypes.data, _threads())
    return W


def uniform01(n: int, seed: int) -> np.ndarray:
    """Symmetric FP32 weights uniform in (0,1), zero diagonal."""
    W = np.empty((n, n), dtype=np.float32)
    _lib().synth_uniform01_f32(seed, n, W.ctypes.data, _threads())
    return W


def mix64(x: int) -> int:
    return int(_lib().synth_mix64(x))


def hash3(seed: int, lo: int, hi: int) -> int:
    return int(_lib().synth_hash(seed, lo, hi))


# ------------------------------------------------------- device generator
def _cuda_lib():
    global _CUDA_LIB
    with _LOCK:
        if _CUDA_LIB is None:
            lib = ctypes.CDLL(build_cuda())
            lib.synth_cuda_euclid_f32.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                  ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_cuda_euclid_f32.restype = ctypes.c_int
            lib.synth_cuda_hash_u32.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p]
            lib.synth_cuda_hash_u32.restype = ctypes.c_int
            lib.synth_cuda_uniform01_f32.argtypes = [ctypes.c_uint64, ctypes.c_int64,
                                                     ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_cuda_uniform01_f32.restype = ctypes.c_int
            lib.synth_cuda_euclid32_f32.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                    ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_cuda_euclid32_f32.restype = ctypes.c_int
            lib.synth_cuda_requests.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                                ctypes.c_void_p]
            lib.synth_cuda_requests.restype = ctypes.c_int
            _CUDA_LIB = lib
    return _CUDA_LIB


def device_euclid(points_dev_ptr: int, n: int, d: int, W_dev_ptr: int, stream: int = 0) -> None:
    """Fill a device n x n FP32 matrix from device FP32 points (same definition)."""
    rc = _cuda_lib().synth_cuda_euclid_f32(points_dev_ptr, n, d, W_dev_ptr, stream)
    if rc != 0:
        raise RuntimeError(f"synth_cuda_euclid_f32 failed: {rc}")


def device_hash_u32(seed: int, n: int, W_dev_ptr: int, stream: int = 0) -> None:
    rc = _cuda_lib().synth_cuda_hash_u32(seed, n, W_dev_ptr, stream)
    if rc != 0:
        raise RuntimeError(f"synth_cuda_hash_u32 failed: {rc}")


def device_euclid32(points_dev_ptr: int, n: int, d: int, W_dev_ptr: int, stream: int = 0) -> None:
    """Device twin of euclid32 (FP32-arithmetic distances)."""
    rc = _cuda_lib().synth_cuda_euclid32_f32(points_dev_ptr, n, d, W_dev_ptr, stream)
    if rc != 0:
        raise RuntimeError(f"synth_cuda_euclid32_f32 failed: {rc}")


REQ_DESC = np.dtype([("slot", "<u8"), ("pts", "<u8"), ("tile0", "<u8"), ("seed", "<u8"),
                     ("n", "<u4"), ("kind", "<u4"), ("d", "<u4"), ("pad", "<u4")])
REQ_TILE = 1024


def request_descs(slots, pts_ptrs, ns, kinds, seeds, d: int = 2):
    """Descriptors of serving requests for device_requests: kind 0 = FP32
    points (euclid32 of the n x d points at pts_ptrs[k]), 1 = hashed uint32
    weights with seeds[k].  Returns (descriptor array, total tiles)."""
    cnt = len(ns)
    desc = np.zeros(cnt, dtype=REQ_DESC)
    nn = np.asarray(ns, dtype=np.int64)
    tiles = (nn * nn + REQ_TILE - 1) // REQ_TILE
    desc["slot"] = np.asarray(slots, dtype=np.uint64)
    desc["pts"] = np.asarray(pts_ptrs, dtype=np.uint64)
    desc["tile0"] = np.concatenate([[0], np.cumsum(tiles)[:-1]]).astype(np.uint64) if cnt else []
    desc["seed"] = np.asarray(seeds, dtype=np.uint64)
    desc["n"] = nn.astype(np.uint32)
    desc["kind"] = np.asarray(kinds, dtype=np.uint32)
    desc["d"] = d
    return desc, int(tiles.sum())


def device_requests(desc_dev_ptr: int, count: int, total_tiles: int, stream: int = 0) -> None:
    """One launch that writes every described request's W into its slot
    (descriptors already in device memory)."""
    rc = _cuda_lib().synth_cuda_requests(desc_dev_ptr, count, total_tiles, stream)
    if rc != 0:
        raise RuntimeError(f"synth_cuda_requests failed: {rc}")


def device_uniform01(seed: int, n: int, W_dev_ptr: int, stream: int = 0) -> None:
    rc = _cuda_lib().synth_cuda_uniform01_f32(seed, n, W_dev_ptr, stream)
    if rc != 0:
        raise RuntimeError(f"synth_cuda_uniform01_f32 failed: {rc}")


# ------------------------------------------------------------ the configs
# Workloads shaped like the paper's (dense complete graphs from point clouds
# and random weights).  Seeds are fixed per workload.
def cfg1_points() -> np.ndarray:
    """n=1000, 2-D, 5-component mixture, means uniform in [0,10]^2, sigma 0.5."""
    return gmm_points(1000, 2, 5, sigma=0.5, seed=1, mean_box=10.0)


def cfg2a_points(n: int = 16384) -> np.ndarray:
    """n=16384 points uniform in [0,1]^2."""
    return uniform_points(n, 2, seed=2)


CFG2B_SEED = 3


def cfg3_points(n: int = 65536) -> np.ndarray:
    """n=65536, 16-D, 32-component mixture, means N(0, 25 I), sigma 1."""
    return gmm_points(n, 16, 32, sigma=1.0, seed=4, mean_std=5.0)


def cfg4_sizes(count: int = 4096, seed: int = 4) -> np.ndarray:
    """Batched sizes n = floor(32 * 64^u), u ~ U[0,1), clipped to [32, 2048]."""
    rng = np.random.default_rng(seed)
    u = rng.random(count)
    n = np.floor(32.0 * np.power(64.0, u)).astype(np.int64)
    return np.clip(n, 32, 2048)


def cfg4_seed(g: int) -> int:
    return 1000 + g
