"""The solve entry point that allocates nothing (appd_solve_noalloc).

It exists for callers that cannot call cudaMalloc -- for example code that
runs inside a memory pool or arena owned by a framework -- and keeps all its
scratch in a fixed 4 MiB device array inside the library, which limits it to
n <= 1024.  The test calls it through the C ABI and compares it with
appd_solve bit for bit (the results are exact), twice in a row, since the
array is shared and keeps the previous call's contents, and with the CPU
oracle, for both orders (minimax and widest paths).  This file is collected
last on purpose."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2407_07058_gb300 import appd


def _cases():
    rng = np.random.default_rng(2024)
    out = [synth.euclid(synth.gmm_points(1000, 2, 5, sigma=0.5, seed=11, mean_box=10.0)),
           synth.hash_u32(1024, seed=12), synth.uniform01(257, seed=13), synth.hash_u32(2, seed=14),
           np.zeros((1, 1), np.float32)]
    ties = rng.integers(0, 3, size=(300, 300)).astype(np.uint32)
    ties = np.triu(ties, 1)
    out.append(np.ascontiguousarray(ties + ties.T))
    return out


def _dev(W):
    return torch.from_numpy(W if W.dtype == np.float32 else W.view(np.int32)).cuda()


@pytest.mark.gpu
def test_noalloc_matches_solve_on_two_calls_in_a_row():
    lib = appd.load()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        for W in _cases():
            n = W.shape[0]
            dt = appd.F32 if W.dtype == np.float32 else appd.U32
            T = _dev(W)
            ref = appd.solve(T)
            out = torch.full_like(T, -1)
            rc = lib.appd_solve_noalloc(T.data_ptr(), n, dt, out.data_ptr(), stream)
            assert rc == 0, appd.STATUS.get(rc, rc)
            torch.cuda.synchronize()
            assert appd.last_device_status() == 0
            assert torch.equal(out, ref), f"call {call}: n={n} differs from appd_solve"
            got = out.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, oracle.appd(W).view(np.uint32)), f"n={n} differs from the oracle"


@pytest.mark.gpu
def test_noalloc_widest_matches_oracle():
    lib = appd.load()
    stream = torch.cuda.current_stream().cuda_stream
    for W in _cases():
        n = W.shape[0]
        dt = (appd.F32 if W.dtype == np.float32 else appd.U32) | appd.WIDEST
        T = _dev(W)
        out = torch.full_like(T, -1)
        assert lib.appd_solve_noalloc(T.data_ptr(), n, dt, out.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert appd.last_device_status() == 0
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.appd(W, widest=True).view(np.uint32)), f"widest n={n}"


@pytest.mark.gpu
def test_noalloc_in_place_and_limit():
    lib = appd.load()
    stream = torch.cuda.current_stream().cuda_stream
    W = synth.uniform01(600, seed=21)
    T = _dev(W)
    ref = appd.solve(T)
    rc = lib.appd_solve_noalloc(T.data_ptr(), 600, appd.F32, T.data_ptr(), stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.equal(T, ref)
    big = torch.zeros((1025, 1025), dtype=torch.float32, device="cuda")
    assert lib.appd_solve_noalloc(big.data_ptr(), 1025, appd.F32, big.data_ptr(), stream) == 2
