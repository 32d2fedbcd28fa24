"""CPU oracle for the all-pairs minimax-path matrix -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline /
reference arm may import this package.  The product (the CUDA library and its
binding) never does; it shares no code with ``appd_oracle.c``.

Functions take a dense symmetric ``numpy`` matrix of dtype float32 or uint32 and
return the matrix of original weight bits in the same dtype (diagonal 0):

- ``appd(W)``: Prim + descending Algorithm 4 (Sections 3 and 5).
- ``appd_ascending(W)``: the ascending alternative of Section 3.
- ``fw(W)``: (min,max) Floyd-Warshall (Section 1, Table 1), n <= 4096.
- ``brute(W)``: all simple paths, Eq. 1-2, n <= 9.
- ``prim(W)``: Prim order and the MST edge codes.
- ``tree_rows(W, mst, sources)``: rows of M by traversing the MST.
- ``prim_rows(W, order, mst, sources)``: rows of M from Prim's visiting order.
- ``points_w(X)``: FP32 edge weights of a point set (fixed-order FMA distance).
- ``insert(M, w)``: warm start, the matrix of G + p from G's (Section 6.1).

Every function takes ``widest=True`` for the widest-path matrix (Section 4.2:
the largest possible smallest edge weight over all paths), computed by the
same routines with the order of every comparison reversed -- a maximum
spanning tree, its edges removed in ascending order.
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

F32, U32 = 0, 1
WIDEST = 2   # flag: reverse the order (widest paths)


def build() -> str:
    """Compile the oracle with gcc (plain C, -O2, no FMA contraction; OpenMP
    only spreads the independent rows of prim_rows and points_w over the
    cores)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liboracle.so")
    src = os.path.join(_HERE, "appd_oracle.c")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fopenmp", "-shared",
                               "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            lib.appd_oracle_alg4.argtypes = [vp, i64, ci, vp, vp]
            lib.appd_oracle_ascending.argtypes = [vp, i64, ci, vp]
            lib.appd_oracle_fw.argtypes = [vp, i64, ci, vp]
            lib.appd_oracle_brute.argtypes = [vp, i64, ci, vp]
            lib.appd_oracle_prim.argtypes = [vp, i64, ci, vp, vp]
            lib.appd_oracle_prim_sym.argtypes = [vp, i64, ci, vp, vp]
            lib.appd_oracle_tree_rows.argtypes = [vp, i64, ci, vp, vp, i64, vp]
            lib.appd_oracle_insert.argtypes = [vp, i64, ci, vp, vp]
            lib.appd_oracle_prim_rows.argtypes = [vp, i64, ci, vp, vp, vp, i64, vp]
            lib.appd_oracle_points_w.argtypes = [vp, i64, ci, vp]
            lib.appd_oracle_set_mutation.argtypes = [ci]
            lib.appd_oracle_set_short_limit.argtypes = [i64]
            lib.appd_oracle_code_ends.argtypes = [vp, i64, i64, vp, vp]
            lib.appd_oracle_order_key.argtypes = [ctypes.c_uint32, ci]
            lib.appd_oracle_order_key.restype = ctypes.c_uint32
            _LIB = lib
    return _LIB


def _prep(W: np.ndarray, widest: bool = False):
    if W.dtype == np.float32:
        dt = F32
    elif W.dtype == np.uint32:
        dt = U32
    else:
        raise TypeError(f"oracle takes float32 or uint32, got {W.dtype}")
    if W.ndim != 2 or W.shape[0] != W.shape[1]:
        raise ValueError("W must be square")
    Wc = np.ascontiguousarray(W)
    return Wc, Wc.shape[0], dt | (WIDEST if widest else 0)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def appd(W: np.ndarray, *, return_fill_count: bool = False, widest: bool = False):
    Wc, n, dt = _prep(W, widest)
    M = np.empty_like(Wc)
    cnt = ctypes.c_int64(0)
    _check(_lib().appd_oracle_alg4(Wc.ctypes.data, n, dt, M.ctypes.data, ctypes.byref(cnt)),
           "appd_oracle_alg4")
    return (M, cnt.value) if return_fill_count else M


def appd_ascending(W: np.ndarray, widest: bool = False) -> np.ndarray:
    Wc, n, dt = _prep(W, widest)
    M = np.empty_like(Wc)
    _check(_lib().appd_oracle_ascending(Wc.ctypes.data, n, dt, M.ctypes.data),
           "appd_oracle_ascending")
    return M


def fw(W: np.ndarray, widest: bool = False) -> np.ndarray:
    Wc, n, dt = _prep(W, widest)
    M = np.empty_like(Wc)
    _check(_lib().appd_oracle_fw(Wc.ctypes.data, n, dt, M.ctypes.data), "appd_oracle_fw")
    return M


def brute(W: np.ndarray, widest: bool = False) -> np.ndarray:
    Wc, n, dt = _prep(W, widest)
    M = np.empty_like(Wc)
    _check(_lib().appd_oracle_brute(Wc.ctypes.data, n, dt, M.ctypes.data), "appd_oracle_brute")
    return M


def prim(W: np.ndarray, widest: bool = False):
    """Return (order, mst_codes): Prim order from vertex 0 and the n-1 edge codes.

    mst_codes[k] = key << 32 | p of the edge that added order[k+1] (with
    widest=True: the maximum spanning tree, key complemented), where the pair
    number p is lo << 16 | hi for n <= 65536 and otherwise the rank of (lo, hi)
    among all pairs in lexicographic order (see ``code_ends``).
    """
    Wc, n, dt = _prep(W, widest)
    order = np.empty(n, dtype=np.uint32)
    mst = np.empty(max(n - 1, 1), dtype=np.uint64)
    _check(_lib().appd_oracle_prim(Wc.ctypes.data, n, dt, mst.ctypes.data, order.ctypes.data),
           "appd_oracle_prim")
    return order, mst[: n - 1]


def prim_sym(W: np.ndarray, widest: bool = False):
    """prim() for a W that is symmetric bit for bit, reading whole rows (the
    same result; sequential reads for the largest matrices)."""
    Wc, n, dt = _prep(W, widest)
    order = np.empty(n, dtype=np.uint32)
    mst = np.empty(max(n - 1, 1), dtype=np.uint64)
    _check(_lib().appd_oracle_prim_sym(Wc.ctypes.data, n, dt, mst.ctypes.data, order.ctypes.data),
           "appd_oracle_prim_sym")
    return order, mst[: n - 1]


def code_ends(codes: np.ndarray, n: int):
    """(lo, hi) endpoint arrays of edge codes of an n-vertex graph."""
    c = np.ascontiguousarray(codes, dtype=np.uint64)
    lo = np.empty(len(c), dtype=np.uint32)
    hi = np.empty(len(c), dtype=np.uint32)
    _check(_lib().appd_oracle_code_ends(c.ctypes.data, len(c), n, lo.ctypes.data, hi.ctypes.data),
           "appd_oracle_code_ends")
    return lo, hi


class short_limit:
    """Context manager: graphs above ``limit`` vertices use the rank form of
    the pair number (tests of that form on small graphs)."""

    def __init__(self, limit: int):
        self.limit = limit

    def __enter__(self):
        _lib().appd_oracle_set_short_limit(self.limit)
        return self

    def __exit__(self, *exc):
        _lib().appd_oracle_set_short_limit(65536)
        return False


def tree_rows(W: np.ndarray, mst: np.ndarray, sources, widest: bool = False) -> np.ndarray:
    Wc, n, dt = _prep(W, widest)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.uint32))
    mst = np.ascontiguousarray(mst, dtype=np.uint64)
    rows = np.empty((len(src), n), dtype=Wc.dtype)
    _check(_lib().appd_oracle_tree_rows(Wc.ctypes.data, n, dt, mst.ctypes.data, src.ctypes.data,
                                        len(src), rows.ctypes.data), "appd_oracle_tree_rows")
    return rows


def prim_rows(W: np.ndarray, order: np.ndarray, mst: np.ndarray, sources,
              widest: bool = False) -> np.ndarray:
    """Rows of M for the given sources, read off Prim's visiting order
    (``order, mst = prim(W)``): M(order[a], order[b]) is the largest of the
    edges that added order[a+1..b].  O(n) per row."""
    Wc, n, dt = _prep(W, widest)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.uint32))
    order = np.ascontiguousarray(order, dtype=np.uint32)
    mst = np.ascontiguousarray(mst, dtype=np.uint64)
    rows = np.empty((len(src), n), dtype=Wc.dtype)
    _check(_lib().appd_oracle_prim_rows(Wc.ctypes.data, n, dt, mst.ctypes.data, order.ctypes.data,
                                        src.ctypes.data, len(src), rows.ctypes.data),
           "appd_oracle_prim_rows")
    return rows


def points_w(X: np.ndarray) -> np.ndarray:
    """FP32 edge weights of the complete graph of a point set: for i != j,
    W(i,j) = sqrt(s) with s accumulated over the coordinates in order as
    s = fma(t, t, s), t = X(i,k) - X(j,k), every step an FP32 rounding."""
    Xc = np.ascontiguousarray(X, dtype=np.float32)
    if Xc.ndim != 2:
        raise ValueError("X must be n x d")
    n, d = Xc.shape
    W = np.empty((n, n), dtype=np.float32)
    _check(_lib().appd_oracle_points_w(Xc.ctypes.data, n, d, W.ctypes.data), "appd_oracle_points_w")
    return W


def insert(M: np.ndarray, w: np.ndarray, widest: bool = False) -> np.ndarray:
    """Warm start (Section 6.1): the matrix of G + p from G's matrix M and the
    weights w of p's edges; p becomes the last index."""
    Mc, n, dt = _prep(M, widest)
    wc = np.ascontiguousarray(np.asarray(w, dtype=Mc.dtype))
    if wc.shape != (n,):
        raise ValueError("w must hold one weight per vertex")
    out = np.empty((n + 1, n + 1), dtype=Mc.dtype)
    _check(_lib().appd_oracle_insert(Mc.ctypes.data, n, dt, wc.ctypes.data, out.ctypes.data),
           "appd_oracle_insert")
    return out


def order_key(bits: int, dtype: int) -> int:
    return int(_lib().appd_oracle_order_key(bits, dtype))


class mutation:
    """Context manager that plants mistake ``k`` in the oracle (tests only)."""

    def __init__(self, k: int):
        self.k = k

    def __enter__(self):
        _lib().appd_oracle_set_mutation(self.k)
        return self

    def __exit__(self, *exc):
        _lib().appd_oracle_set_mutation(0)
        return False
