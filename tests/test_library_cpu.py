"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol declared in include/appd.h, and rejects bad arguments before touching
the GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2407_07058_gb300 import _build, appd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "appd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(appd_\w+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(appd.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    lib = appd.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings():
    lib = appd.load()
    for code, name in appd.STATUS.items():
        assert lib.appd_status_str(code).decode() == name


def test_argument_errors_need_no_gpu():
    lib = appd.load()
    fake = ctypes.c_void_p(0x1000)      # never dereferenced: rejected first
    fake2 = ctypes.c_void_p(0x2000)
    assert lib.appd_solve(None, 4, 0, fake, None) == 1          # null W
    assert lib.appd_solve(fake, 4, 0, None, None) == 1          # null M
    assert lib.appd_solve(fake, -1, 0, fake2, None) == 1        # n < 0
    assert lib.appd_solve(fake, 4, 7, fake2, None) == 1         # bad dtype
    assert lib.appd_solve(fake, 92683, 0, fake2, None) == 2     # too large (n (n-1) / 2 > 2^32)
    assert lib.appd_solve(fake, 0, 0, fake2, None) == 0         # n == 0: no-op
    # partial overlap of M and W (M == W exactly is allowed)
    assert lib.appd_solve(ctypes.c_void_p(0x10000), 64, 0, ctypes.c_void_p(0x10000 + 64), None) == 8
    assert lib.appd_solve_alg4(fake, 92683, 1, fake2, None) == 2
    assert lib.appd_mst(None, 4, 0, fake, None) == 1
    assert lib.appd_mst(fake, 65537, 0, fake2, None) == 2       # 16-bit endpoints in this format
    assert lib.appd_mst_edges(fake, 92683, 0, fake2, fake2, fake2, None) == 2
    assert lib.appd_mst_edges(fake, 10, 0, None, fake2, fake2, None) == 1
    assert lib.appd_leaf_order(fake, 92683, 0, fake2, fake2, None) == 2
    assert lib.appd_insert_vertex(fake, 92682, 0, fake2, ctypes.c_void_p(0x10 << 40), None) == 2
    assert lib.appd_solve_points(fake, 92683, 2, 0, fake2, None) == 2
    assert lib.appd_check_symmetric(None, 4, 0, None) == 1
    assert lib.appd_solve_batched(None, None, None, None, None, -1, None) == 1
    assert lib.appd_batched_get_tuning(None, None, None) == 1


def test_tuning_readback_needs_no_gpu():
    appd.batched_tuning(1, 128, 1024)
    appd.batched_prim_max(64)
    try:
        assert appd.get_batched_tuning() == {"ctas_per_sm": 1, "fill_rows": 128, "n_split": 1024,
                                             "prim_max": 64}
    finally:
        appd.batched_tuning()
        appd.batched_prim_max()
    assert appd.get_batched_tuning() == {"ctas_per_sm": 1, "fill_rows": 256, "n_split": 2048,
                                         "prim_max": 256}
    lib = appd.load()
    assert lib.appd_batched_prim_max(513) == 1 and lib.appd_batched_prim_max(-1) == 1


def test_build_is_in_tree_for_sm103a():
    assert _build.lib_path().startswith(os.path.join(ROOT, "paper_2407_07058_gb300"))
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
