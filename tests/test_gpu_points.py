"""GPU parity of the point-set solve (appd_solve_points) against the oracle.

The library never forms W: it computes each edge weight from the coordinates
where the MST reads it.  The oracle forms W with its own routine
(oracle.points_w: the FP32 fixed-order definition, pinned in
tests/test_oracle_pins.py against exact rational arithmetic) and solves it
with Prim + Algorithm 4, so the two sides share nothing but the points.
Results are compared bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2407_07058_gb300 import appd
from tests.test_gpu_parity import assert_bits

pytestmark = pytest.mark.gpu


def solve_points(X: np.ndarray, widest: bool = False) -> np.ndarray:
    M = appd.solve_points(torch.from_numpy(np.ascontiguousarray(X)).cuda(), widest=widest)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    return M.cpu().numpy()


def ref_points(X: np.ndarray, widest: bool = False) -> np.ndarray:
    return oracle.appd(oracle.points_w(X), widest=widest)


def _points(n, d, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "gmm":
        return synth.gmm_points(n, d, 5, sigma=0.5, seed=seed, mean_box=10.0)
    if kind == "grid":       # integer grid: many equal distances
        return rng.integers(0, 4, size=(n, d)).astype(np.float32)
    if kind == "dup":        # repeated points: zero-weight edges and ties
        base = rng.random((max(1, n // 4), d)).astype(np.float32)
        return np.ascontiguousarray(base[rng.integers(0, len(base), size=n)])
    return rng.standard_normal((n, d)).astype(np.float32) * 100.0


CASES = [(1, 2), (2, 1), (3, 3), (5, 2), (31, 16), (32, 4), (33, 5), (100, 8), (257, 2), (1000, 16),
         (1031, 3), (2049, 17), (4099, 2), (3000, 32)]


@pytest.mark.parametrize("n,d", CASES)
@pytest.mark.parametrize("kind", ["gmm", "grid", "dup", "wide"])
def test_points_parity(n, d, kind):
    X = _points(n, d, kind, 7000 + n + d)
    assert_bits(solve_points(X), ref_points(X), f"points n={n} d={d} {kind}")


@pytest.mark.parametrize("n,d", [(5, 2), (257, 16), (1031, 3), (4099, 2)])
@pytest.mark.parametrize("kind", ["gmm", "grid"])
def test_points_widest_parity(n, d, kind):
    X = _points(n, d, kind, 8000 + n)
    assert_bits(solve_points(X, widest=True), ref_points(X, widest=True), f"widest points n={n} d={d}")


@pytest.mark.parametrize("d", [2, 16])
def test_points_n16384(d):
    X = synth.cfg2a_points() if d == 2 else synth.cfg3_points(16384)
    assert_bits(solve_points(X), ref_points(X), f"points n=16384 d={d}")


def test_points_full_size_every_row():
    """The 16-D mixture points of the n = 65536 workload, every row: W is
    formed on the host by the oracle and the rows are read off Prim's order."""
    n = 65536
    X = synth.cfg3_points(n)
    T = torch.from_numpy(X).cuda()
    M = torch.empty((n, n), dtype=torch.float32, device="cuda")
    for _ in range(2):
        appd.solve_points(T, out=M)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    W = oracle.points_w(X)
    order, mst = oracle.prim_sym(W)   # the definition is symmetric bit for bit
    for r0 in range(0, n, 4096):
        ref = oracle.prim_rows(W, order, mst, np.arange(r0, r0 + 4096))
        assert_bits(M[r0: r0 + 4096].cpu().numpy(), ref, f"points n={n} rows {r0}..")


def test_points_argument_errors():
    lib = appd.load()
    X = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    M = torch.empty((10, 10), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.appd_solve_points(X.data_ptr(), 10, 0, appd.F32, M.data_ptr(), st) == 1
    assert lib.appd_solve_points(X.data_ptr(), 10, 33, appd.F32, M.data_ptr(), st) == 1
    assert lib.appd_solve_points(X.data_ptr(), 10, 4, appd.U32, M.data_ptr(), st) == 1
    assert lib.appd_solve_points(X.data_ptr(), 92683, 4, appd.F32, M.data_ptr(), st) == 2
    assert lib.appd_solve_points(X.data_ptr(), 10, 4, appd.F32, X.data_ptr(), st) == 8
    assert lib.appd_solve_points(X.data_ptr(), 0, 4, appd.F32, M.data_ptr(), st) == 0
