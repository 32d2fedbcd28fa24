"""Python binding of the APPD C ABI (include/appd.h).

Argument marshalling only: every step of a solve runs in the CUDA library
``_build/libappd.so``.  Tensors must live on a CUDA device; there is no CPU
fallback, and loading fails loudly if the library cannot be built or loaded.

dtype mapping: ``torch.float32`` -> APPD_F32; ``torch.int32`` / ``torch.uint32``
-> APPD_U32 (the 32 bits are read as an unsigned integer).
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import _build

F32, U32 = 0, 1
WIDEST = 2                       # dtype bit: widest paths (Section 4.2)
F32_WIDEST, U32_WIDEST = 2, 3
STATUS = {0: "APPD_OK", 1: "APPD_ERR_INVALID", 2: "APPD_ERR_TOO_LARGE", 3: "APPD_ERR_NOMEM",
          4: "APPD_ERR_CUDA", 5: "APPD_ERR_ASYMMETRIC", 6: "APPD_ERR_TIMEOUT", 7: "APPD_ERR_BUSY",
          8: "APPD_ERR_ALIAS", 9: "APPD_ERR_NOT_FOUND", 10: "APPD_ERR_INTERNAL"}

# every symbol that include/appd.h declares
EXPORTS = ["appd_status_str", "appd_solve", "appd_solve_points", "appd_solve_alg4", "appd_solve_host",
           "appd_solve_host_async", "appd_solve_host_wait", "appd_solve_noalloc", "appd_insert_vertex", "appd_insert_vertex_tree", "appd_mst",
           "appd_mst_edges", "appd_leaf_order",
           "appd_solve_batched", "appd_batched_tuning", "appd_batched_autotune",
           "appd_batched_get_tuning", "appd_batched_prim_max", "appd_batched_get_prim_max",
           "appd_check_symmetric",
           "appd_last_device_status", "appd_probe_bounded_wait", "appd_release_workspaces",
           "appd_debug_mark_failed", "appd_profile_begin",
           "appd_profile_end", "appd_server_create",
           "appd_server_submit", "appd_server_submit_many", "appd_server_commit",
           "appd_server_commit_many", "appd_server_poll", "appd_server_release",
           "appd_server_release_many", "appd_server_destroy"]

_LOCK = threading.Lock()
_LIB = None


class AppdError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


def load(build_if_missing: bool = True):
    """Load libappd.so (building it first if it is missing or stale)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if build_if_missing and _build.is_stale():
            _build.build()
        lib = ctypes.CDLL(_build.lib_path())
        vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        ci = ctypes.c_int
        sig = {
            "appd_solve": [vp, i64, ci, vp, vp],
            "appd_solve_points": [vp, i64, i32, ci, vp, vp],
            "appd_solve_alg4": [vp, i64, ci, vp, vp],
            "appd_solve_host": [vp, i64, ci, vp, vp],
            "appd_solve_host_async": [vp, i64, ci, vp, vp],
            "appd_solve_host_wait": [vp],
            "appd_insert_vertex": [vp, i64, ci, vp, vp, vp],
            "appd_insert_vertex_tree": [vp, vp, vp, i64, ci, vp, vp, vp, vp, vp, vp],
            "appd_solve_noalloc": [vp, i64, ci, vp, vp],
            "appd_mst": [vp, i64, ci, vp, vp],
            "appd_mst_edges": [vp, i64, ci, vp, vp, vp, vp],
            "appd_leaf_order": [vp, i64, ci, vp, vp, vp],
            "appd_solve_batched": [vp, vp, vp, vp, vp, i32, vp],
            "appd_batched_tuning": [i32, i32, i64],
            "appd_batched_autotune": [ctypes.c_char_p, vp],
            "appd_batched_get_tuning": [ctypes.POINTER(i32), ctypes.POINTER(i32),
                                        ctypes.POINTER(i64)],
            "appd_batched_prim_max": [i32],
            "appd_batched_get_prim_max": [ctypes.POINTER(i32)],
            "appd_check_symmetric": [vp, i64, ci, vp],
            "appd_last_device_status": [vp],
            "appd_probe_bounded_wait": [i32, vp],
            "appd_release_workspaces": [],
            "appd_server_create": [ctypes.c_size_t, i32, ctypes.POINTER(vp)],
            "appd_server_submit": [vp, i64, ci, vp, ctypes.POINTER(u64), ctypes.POINTER(vp)],
            "appd_server_commit": [vp, u64, vp],
            "appd_server_submit_many": [vp, i32, vp, vp, vp, vp, vp, ctypes.POINTER(i32)],
            "appd_server_commit_many": [vp, i32, vp, vp],
            "appd_server_poll": [vp, vp, vp, i32, ctypes.POINTER(i32)],
            "appd_server_release": [vp, u64, vp],
            "appd_server_release_many": [vp, i32, vp, vp],
            "appd_server_destroy": [vp],
            "appd_debug_mark_failed": [],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ci
        lib.appd_profile_begin.argtypes = []
        lib.appd_profile_begin.restype = i32
        lib.appd_profile_end.argtypes = [ctypes.POINTER(ctypes.c_double), i32]
        lib.appd_profile_end.restype = i32
        lib.appd_status_str.argtypes = [ci]
        lib.appd_status_str.restype = ctypes.c_char_p
        _LIB = lib
        return lib


def _check(code: int, what: str):
    if code != 0:
        raise AppdError(code, what)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype in (torch.int32, getattr(torch, "uint32", torch.int32)):
        return U32
    raise TypeError(f"unsupported dtype {t.dtype}: use float32, int32 or uint32")


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _square_cuda(W):
    if not W.is_cuda:
        raise ValueError("W must be a CUDA tensor (no CPU path)")
    if W.dim() != 2 or W.shape[0] != W.shape[1] or not W.is_contiguous():
        raise ValueError("W must be a contiguous square matrix")
    return W.shape[0]


def solve(W, out=None, stream=None, alg4: bool = False, widest: bool = False):
    """APPD matrix of W (n x n, symmetric) on W's device; returns M (same dtype).

    widest=True gives the widest-path matrix instead (largest smallest edge)."""
    import torch
    n = _square_cuda(W)
    dt = _dtype_code(W) | (WIDEST if widest else 0)
    M = torch.empty_like(W) if out is None else out
    fn = load().appd_solve_alg4 if alg4 else load().appd_solve
    with torch.cuda.device(W.device):
        _check(fn(W.data_ptr(), n, dt, M.data_ptr(), _stream_ptr(stream)), "appd_solve")
    return M


def solve_points(X, out=None, stream=None, widest: bool = False):
    """APPD matrix of the complete graph of the points X (n x d FP32, CUDA),
    edge weights computed on the fly in FP32 (see appd.h); returns M (n x n)."""
    import torch
    if not X.is_cuda:
        raise ValueError("X must be a CUDA tensor (no CPU path)")
    if X.dim() != 2 or X.dtype != torch.float32 or not X.is_contiguous():
        raise ValueError("X must be a contiguous n x d float32 matrix")
    n, d = X.shape
    M = torch.empty((n, n), dtype=torch.float32, device=X.device) if out is None else out
    dt = F32 | (WIDEST if widest else 0)
    with torch.cuda.device(X.device):
        _check(load().appd_solve_points(X.data_ptr(), n, d, dt, M.data_ptr(), _stream_ptr(stream)),
               "appd_solve_points")
    return M


def solve_alg4(W, out=None, stream=None, widest: bool = False):
    return solve(W, out=out, stream=stream, alg4=True, widest=widest)


def solve_host(W: np.ndarray, stream=None, widest: bool = False) -> np.ndarray:
    """APPD of a host matrix through appd_solve_host (copies inside the call)."""
    Wc = np.ascontiguousarray(W)
    if Wc.dtype == np.float32:
        dt = F32
    elif Wc.dtype in (np.uint32, np.int32):
        dt = U32
    else:
        raise TypeError(f"unsupported dtype {Wc.dtype}")
    dt |= WIDEST if widest else 0
    M = np.empty_like(Wc)
    _check(load().appd_solve_host(Wc.ctypes.data, Wc.shape[0], dt, M.ctypes.data,
                                  _stream_ptr(stream)), "appd_solve_host")
    return M


def solve_host_ptr(W_ptr: int, n: int, dt: int, M_ptr: int, stream=None):
    """appd_solve_host on raw host pointers (e.g. pinned buffers)."""
    _check(load().appd_solve_host(W_ptr, n, dt, M_ptr, _stream_ptr(stream)), "appd_solve_host")


def insert_vertex(M, w, out=None, stream=None, widest: bool = False):
    """Warm start (Section 6.1): the (n+1) x (n+1) matrix of G + p from G's
    matrix M (n x n, from solve) and the n weights w of p's edges."""
    import torch
    n = _square_cuda(M)
    if not w.is_cuda or w.numel() != n or w.dtype != M.dtype:
        raise ValueError("w must be a CUDA vector of n weights of M's dtype")
    Mo = torch.empty((n + 1, n + 1), dtype=M.dtype, device=M.device) if out is None else out
    dt = _dtype_code(M) | (WIDEST if widest else 0)
    with torch.cuda.device(M.device):
        _check(load().appd_insert_vertex(M.data_ptr(), n, dt, w.contiguous().data_ptr(), Mo.data_ptr(),
                                         _stream_ptr(stream)), "appd_insert_vertex")
    return Mo


def insert_vertex_tree(tree, w, n: int, dtype, out=None, tree_out: bool = True, stream=None,
                       widest: bool = False):
    """Warm start through the tree: tree = (keys, lo, hi) of G (mst_edges),
    w the n weights of the new vertex's edges (CUDA, dtype float32 or int32).
    Returns (M_out, new tree or None)."""
    import torch
    keys, lo, hi = tree
    if not w.is_cuda or w.numel() != n:
        raise ValueError("w must be a CUDA vector of n weights")
    dev = w.device
    Mo = torch.empty((n + 1, n + 1), dtype=w.dtype, device=dev) if out is None else out
    nt = None
    if tree_out:
        nt = tuple(torch.empty(max(n, 1), dtype=torch.int32, device=dev) for _ in range(3))
    dt = (F32 if dtype == torch.float32 else U32) | (WIDEST if widest else 0)
    ptr = lambda t: t.data_ptr() if t is not None else None
    with torch.cuda.device(dev):
        _check(load().appd_insert_vertex_tree(ptr(keys), ptr(lo), ptr(hi), n, dt, w.contiguous().data_ptr(),
                                              Mo.data_ptr(), *(ptr(t) for t in (nt or (None,) * 3)),
                                              _stream_ptr(stream)), "appd_insert_vertex_tree")
    if nt is not None:
        nt = tuple(t[:n] for t in nt)
    return Mo, nt


def solve_host_async_ptr(W_ptr: int, n: int, dt: int, M_ptr: int, stream=None):
    """appd_solve_host_async on raw host pointers: enqueue and return (see
    solve_host_wait before reading M)."""
    _check(load().appd_solve_host_async(W_ptr, n, dt, M_ptr, _stream_ptr(stream)),
           "appd_solve_host_async")


def solve_host_wait(stream=None):
    """Make the stream wait for every pipelined host call's copy back."""
    _check(load().appd_solve_host_wait(_stream_ptr(stream)), "appd_solve_host_wait")


def mst(W, stream=None, widest: bool = False):
    """The n-1 MST edges as int64 values key<<32 | lo<<16 | hi (order unspecified);
    widest=True: the maximum spanning tree, keys complemented."""
    import torch
    n = _square_cuda(W)
    E = torch.empty(max(n - 1, 1), dtype=torch.int64, device=W.device)
    dt = _dtype_code(W) | (WIDEST if widest else 0)
    with torch.cuda.device(W.device):
        _check(load().appd_mst(W.data_ptr(), n, dt, E.data_ptr(), _stream_ptr(stream)), "appd_mst")
    return E[: n - 1]


def mst_edges(W, stream=None, widest: bool = False):
    """The n-1 MST edges as (keys, lo, hi) int32 tensors (the order key of the
    edge's weight and its endpoints lo < hi), for any n the library takes."""
    import torch
    n = _square_cuda(W)
    m = max(n - 1, 1)
    keys, lo, hi = (torch.empty(m, dtype=torch.int32, device=W.device) for _ in range(3))
    dt = _dtype_code(W) | (WIDEST if widest else 0)
    with torch.cuda.device(W.device):
        _check(load().appd_mst_edges(W.data_ptr(), n, dt, keys.data_ptr(), lo.data_ptr(), hi.data_ptr(),
                                     _stream_ptr(stream)), "appd_mst_edges")
    return keys[: n - 1], lo[: n - 1], hi[: n - 1]


def leaf_order(W, stream=None, widest: bool = False):
    """(pos, gap): leaf position of each vertex and the n-1 merge-height keys."""
    import torch
    n = _square_cuda(W)
    pos = torch.empty(n, dtype=torch.int32, device=W.device)
    gap = torch.empty(max(n - 1, 1), dtype=torch.int32, device=W.device)
    dt = _dtype_code(W) | (WIDEST if widest else 0)
    with torch.cuda.device(W.device):
        _check(load().appd_leaf_order(W.data_ptr(), n, dt, pos.data_ptr(),
                                      gap.data_ptr(), _stream_ptr(stream)), "appd_leaf_order")
    return pos, gap[: n - 1]


def solve_batched(Wflat, offsets, ns, dts=None, out=None, stream=None):
    """Many graphs: graph g is Wflat[offsets[g] : offsets[g] + ns[g]**2] (row-major).

    dts[g] is F32, U32, F32_WIDEST or U32_WIDEST (None: all F32)."""
    import torch
    if not Wflat.is_cuda:
        raise ValueError("Wflat must be a CUDA tensor")
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nn = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
    dd = None if dts is None else np.ascontiguousarray(np.asarray(dts, dtype=np.uint8))
    M = torch.empty_like(Wflat) if out is None else out
    with torch.cuda.device(Wflat.device):
        _check(load().appd_solve_batched(off.ctypes.data, Wflat.data_ptr(), nn.ctypes.data,
                                         None if dd is None else dd.ctypes.data, M.data_ptr(),
                                         len(nn), _stream_ptr(stream)), "appd_solve_batched")
    return M


def check_symmetric(W, stream=None) -> bool:
    n = _square_cuda(W)
    code = load().appd_check_symmetric(W.data_ptr(), n, _dtype_code(W), _stream_ptr(stream))
    if code == 5:
        return False
    _check(code, "appd_check_symmetric")
    return True


def last_device_status(stream=None) -> int:
    return int(load().appd_last_device_status(_stream_ptr(stream)))


PHASES = ["rowmin", "boruvka_step", "contract_w", "contract_c", "leaf_order", "fill", "batched"]


def profile_begin():
    load().appd_profile_begin()


def profile_end() -> dict:
    """Per-phase device ms since profile_begin, kernel launch count, c1."""
    buf = (ctypes.c_double * 9)()
    k = load().appd_profile_end(buf, 9)
    vals = [buf[i] for i in range(k)]
    out = {name: vals[i] for i, name in enumerate(PHASES)}
    out["launches"] = int(vals[7])
    out["c1"] = int(vals[8])
    return out


def batched_tuning(ctas_per_sm: int = 1, fill_rows: int = 256, n_split: int = 2048):
    _check(load().appd_batched_tuning(ctas_per_sm, fill_rows, n_split), "appd_batched_tuning")


def probe_bounded_wait(limit_ms: int = 200, stream=None):
    """Run a grid-barrier wait out on purpose (bounded; see appd.h)."""
    _check(load().appd_probe_bounded_wait(limit_ms, _stream_ptr(stream)), "appd_probe_bounded_wait")


def batched_autotune(cache_path: str | None = None, stream=None) -> dict:
    """Search the batched path's parameters on this GPU (cached in cache_path)."""
    arg = None if cache_path is None else cache_path.encode()
    _check(load().appd_batched_autotune(arg, _stream_ptr(stream)), "appd_batched_autotune")
    return get_batched_tuning()


def get_batched_tuning() -> dict:
    a, b, c, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    _check(load().appd_batched_get_tuning(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "appd_batched_get_tuning")
    _check(load().appd_batched_get_prim_max(ctypes.byref(d)), "appd_batched_get_prim_max")
    return {"ctas_per_sm": a.value, "fill_rows": b.value, "n_split": c.value, "prim_max": d.value}


def batched_prim_max(prim_max: int = 256):
    """Largest batched graph solved by one warp with Prim (0..512)."""
    _check(load().appd_batched_prim_max(prim_max), "appd_batched_prim_max")


def release_workspaces():
    _check(load().appd_release_workspaces(), "appd_release_workspaces")


def debug_mark_failed():
    """Set the failure flag of every control block the library keeps on the
    current device, as a failed earlier solve would (test hook, see appd.h)."""
    _check(load().appd_debug_mark_failed(), "appd_debug_mark_failed")


class _DevPtr:
    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n, n), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def device_view(ptr: int, n: int, dt: int):
    """A torch tensor viewing an n x n matrix at a raw device pointer (e.g. a
    server slot); float32 for F32, int32 for U32.  No copy."""
    import torch
    return torch.as_tensor(_DevPtr(ptr, n, "<f4" if dt == F32 else "<i4"), device="cuda")


class Server:
    """Continuous-batching solve server (appd_server_* entry points)."""

    def __init__(self, budget_bytes: int, max_inflight: int = 4096):
        self._h = ctypes.c_void_p()
        _check(load().appd_server_create(budget_bytes, max_inflight, ctypes.byref(self._h)),
               "appd_server_create")

    def submit(self, n: int, dt: int, stream=None):
        """Returns (req_id, W_slot_ptr) or None when admission is refused (busy).
        Fill the slot on `stream` (default: the current stream)."""
        rid = ctypes.c_uint64()
        slot = ctypes.c_void_p()
        code = load().appd_server_submit(self._h, n, dt, _stream_ptr(stream), ctypes.byref(rid),
                                         ctypes.byref(slot))
        if code == 7:
            return None
        _check(code, "appd_server_submit")
        return rid.value, slot.value

    def submit_many(self, ns, dts, stream=None):
        """Admit the longest prefix of the requests (ns[k], dts[k]) that fits;
        returns (ids, slot pointers) as numpy arrays of the admitted prefix."""
        nn = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
        dd = np.ascontiguousarray(np.asarray(dts, dtype=np.uint8))
        cnt = len(nn)
        ids = np.zeros(max(cnt, 1), dtype=np.uint64)
        slots = np.zeros(max(cnt, 1), dtype=np.uint64)
        k = ctypes.c_int32()
        code = load().appd_server_submit_many(self._h, cnt, nn.ctypes.data, dd.ctypes.data,
                                               _stream_ptr(stream), ids.ctypes.data,
                                               slots.ctypes.data, ctypes.byref(k))
        if code != 7:
            _check(code, "appd_server_submit_many")
        return ids[: k.value], slots[: k.value]

    def commit(self, rid: int, stream=None):
        """Queue the request; its W is complete after the work already on
        `stream` (default: the current stream)."""
        _check(load().appd_server_commit(self._h, rid, _stream_ptr(stream)), "appd_server_commit")

    def commit_many(self, ids, stream=None):
        ii = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
        _check(load().appd_server_commit_many(self._h, len(ii), ii.ctypes.data, _stream_ptr(stream)),
               "appd_server_commit_many")

    def poll(self, cap: int = 1024):
        ids = (ctypes.c_uint64 * cap)()
        ptrs = (ctypes.c_void_p * cap)()
        k = ctypes.c_int32()
        _check(load().appd_server_poll(self._h, ids, ptrs, cap, ctypes.byref(k)), "appd_server_poll")
        return [(ids[i], ptrs[i]) for i in range(k.value)]

    def poll_arrays(self, cap: int = 4096):
        """poll() as numpy arrays (ids, M pointers)."""
        ids = np.zeros(cap, dtype=np.uint64)
        ptrs = np.zeros(cap, dtype=np.uint64)
        k = ctypes.c_int32()
        _check(load().appd_server_poll(self._h, ids.ctypes.data, ptrs.ctypes.data, cap,
                                       ctypes.byref(k)), "appd_server_poll")
        return ids[: k.value], ptrs[: k.value]

    def release(self, rid: int, stream=None):
        """Free the request's slots after the work already on `stream` (its
        reads of M) has run."""
        _check(load().appd_server_release(self._h, rid, _stream_ptr(stream)), "appd_server_release")

    def release_many(self, ids, stream=None):
        ii = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
        _check(load().appd_server_release_many(self._h, len(ii), ii.ctypes.data,
                                                _stream_ptr(stream)), "appd_server_release_many")

    def close(self):
        if self._h:
            _check(load().appd_server_destroy(self._h), "appd_server_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
