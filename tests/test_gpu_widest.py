"""GPU parity of the widest-path matrix (Section 4.2) against the oracle.

The widest dtypes run every comparison of the pipeline in the reversed
order (maximum spanning tree, fill by the smallest edge on the tree path);
the oracle computes the same matrix with its own routines in the reversed
order, pinned in tests/test_oracle_widest.py.  Bit-exact, as for minimax.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2407_07058_gb300 import appd
from tests.test_gpu_parity import _batch, assert_bits, from_dev, special_values, to_dev
from tests.test_oracle_pins import sym_random

pytestmark = pytest.mark.gpu


def solve_widest(W: np.ndarray, alg4=False) -> np.ndarray:
    M = appd.solve(to_dev(W), alg4=alg4, widest=True)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    return from_dev(M, W)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 127, 257, 1000, 1031])
@pytest.mark.parametrize("kind", ["f32", "ties", "special"])
def test_widest_parity(n, kind):
    rng = np.random.default_rng(5000 + n)
    if kind == "f32":
        W = sym_random(n, rng, np.float32)
    elif kind == "ties":
        W = sym_random(n, rng, np.uint32, "ties")
    else:
        W = special_values(n, rng)
    assert_bits(solve_widest(W), oracle.appd(W, widest=True), f"widest n={n} {kind}")


@pytest.mark.parametrize("n", [3, 257, 1000])
def test_widest_alg4_form(n):
    rng = np.random.default_rng(17 + n)
    W = sym_random(n, rng, np.float32)
    assert_bits(solve_widest(W, alg4=True), oracle.appd(W, widest=True), f"widest alg4 n={n}")


@pytest.mark.parametrize("n", [2, 100, 1001, 4099])
def test_maximum_spanning_tree_edge_set(n):
    W = synth.hash_u32(n, seed=n) if n % 2 else synth.uniform01(n, seed=n)
    _, ref = oracle.prim(W, widest=True)
    E = appd.mst(to_dev(W), widest=True).cpu().numpy().view(np.uint64)
    assert np.array_equal(np.sort(E), np.sort(ref))


def test_widest_is_negated_minimax_of_negated_weights_on_device():
    W = synth.euclid(synth.uniform_points(3000, 2, seed=21))
    flip = np.uint32(0x80000000)
    Wn = (W.view(np.uint32) ^ flip).view(np.float32)
    Mw = solve_widest(W).view(np.uint32)
    Mn = appd.solve(to_dev(Wn))
    torch.cuda.synchronize()
    ref = from_dev(Mn, Wn).view(np.uint32) ^ flip
    off = ~np.eye(W.shape[0], dtype=bool)
    assert np.array_equal(Mw[off], ref[off])


def test_widest_config2a_n16384():
    W = synth.euclid(synth.cfg2a_points())
    assert_bits(solve_widest(W), oracle.appd(W, widest=True), "widest n=16384")


def test_batched_mixed_minimax_and_widest():
    sizes = [2, 37, 300, 2048, 2049, 64, 999, 5]
    dts = [appd.F32_WIDEST, appd.U32, appd.U32_WIDEST, appd.F32_WIDEST, appd.U32_WIDEST, appd.F32,
           appd.F32_WIDEST, appd.U32_WIDEST]
    Ws, offs, flat = _batch(sizes, [d & 1 for d in dts], seed0=300)
    T = torch.from_numpy(flat.view(np.int32)).cuda()
    M = appd.solve_batched(T, offs, sizes, dts=dts)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    Mh = M.cpu().numpy().view(np.uint32)
    for g, (W, n, d) in enumerate(zip(Ws, sizes, dts)):
        got = Mh[offs[g]: offs[g] + n * n].reshape(n, n).view(W.dtype)
        assert_bits(got, oracle.appd(W, widest=bool(d & appd.WIDEST)), f"batched graph {g} dt={d}")


def test_widest_host_entry_and_noalloc():
    W = synth.uniform01(700, seed=7)
    ref = oracle.appd(W, widest=True)
    assert_bits(appd.solve_host(W, widest=True), ref, "widest host")
    lib = appd.load()
    T = to_dev(W)
    out = torch.empty_like(T)
    rc = lib.appd_solve_noalloc(T.data_ptr(), 700, appd.F32_WIDEST, out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert_bits(from_dev(out, W), ref, "widest noalloc")


def test_widest_config2b_n16384_ties():
    W = synth.hash_u32(16384, seed=synth.CFG2B_SEED)
    assert_bits(solve_widest(W), oracle.appd(W, widest=True), "widest n=16384 uint32 ties")
