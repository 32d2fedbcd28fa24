"""Solves above 65536 vertices, where an edge's endpoints no longer fit 16
bits each and the packed edge carries the pair's rank among all pairs in
(lo, hi) order instead (the same strict order (key, lo, hi)).

Both checks compare every row with the oracle (rows read off Prim's order,
the oracle's own pair numbering) and the whole MST edge set, at

- n = 92682, the largest n the 32-bit pair rank allows: FP32 distances of
  16-D mixture points (W and M together 68.7 GB on the device);
- n = 70001 uint32 weights with heavy ties: n odd, so rows are not 16-byte
  aligned and the unaligned forms of round 1 and the level-0 contraction run;
- n = 65540 FP32 mixture distances: rows 16-byte aligned and C_1 small enough
  for the bulk-copy contraction, so its fold forms pair ranks (and compares
  raw bits: no weight is negative).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2407_07058_gb300 import appd
from tests.test_gpu_parity import assert_bits

pytestmark = pytest.mark.gpu

ROW_BLOCK = 4096


def _check(W: torch.Tensor, M: torch.Tensor, Wh: np.ndarray, what: str):
    n = Wh.shape[0]
    keys, lo, hi = appd.mst_edges(W)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    got = np.stack([keys.cpu().numpy().view(np.uint32), lo.cpu().numpy().view(np.uint32),
                    hi.cpu().numpy().view(np.uint32)], axis=1).astype(np.uint64)
    order, mst = oracle.prim_sym(Wh)   # W is symmetric by construction
    rlo, rhi = oracle.code_ends(mst, n)
    ref = np.stack([(mst >> 32), rlo, rhi], axis=1).astype(np.uint64)
    key = lambda a: a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]
    assert np.array_equal(key(got), key(ref)), f"{what}: MST edge sets differ"
    for r0 in range(0, n, ROW_BLOCK):
        r1 = min(n, r0 + ROW_BLOCK)
        refr = oracle.prim_rows(Wh, order, mst, np.arange(r0, r1))
        assert_bits(M[r0:r1].cpu().numpy().view(refr.dtype), refr, f"{what} rows {r0}..{r1 - 1}")


def test_largest_n_gmm16_every_row():
    n = 92682
    st = torch.cuda.current_stream().cuda_stream
    pts = torch.from_numpy(synth.gmm_points(n, 16, 32, sigma=1.0, seed=4, mean_std=5.0)).cuda()
    W = torch.empty((n, n), dtype=torch.float32, device="cuda")
    synth.device_euclid(pts.data_ptr(), n, 16, W.data_ptr(), st)
    M = torch.empty_like(W)
    for _ in range(2):
        appd.solve(W, out=M)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    assert int(torch.count_nonzero(torch.diagonal(M))) == 0
    _check(W, M, W.cpu().numpy(), f"n={n} gmm16")


def test_aligned_n_above_16_bits_bulk_copy_contraction_every_row():
    n = 65540
    st = torch.cuda.current_stream().cuda_stream
    pts = torch.from_numpy(synth.gmm_points(n, 16, 32, sigma=1.0, seed=6, mean_std=5.0)).cuda()
    W = torch.empty((n, n), dtype=torch.float32, device="cuda")
    synth.device_euclid(pts.data_ptr(), n, 16, W.data_ptr(), st)
    M = appd.solve(W)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    _check(W, M, W.cpu().numpy(), f"n={n} gmm16 aligned")


def test_odd_n_above_16_bits_uint32_ties_every_row():
    n = 70001
    W = torch.empty((n, n), dtype=torch.int32, device="cuda")
    synth.device_hash_u32(71, n, W.data_ptr(), torch.cuda.current_stream().cuda_stream)
    M = appd.solve(W)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    assert appd.check_symmetric(M)
    _check(W, M, W.cpu().numpy().view(np.uint32), f"n={n} u32 ties")


def test_limits_above_16_bits():
    lib = appd.load()
    W = torch.zeros(16, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.appd_solve(W.data_ptr(), 92683, 0, W.data_ptr(), st) == 2
    assert lib.appd_mst(W.data_ptr(), 65537, 0, W.data_ptr(), st) == 2
