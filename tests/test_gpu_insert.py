"""GPU warm start (Section 6.1, appd_insert_vertex) against the oracle: the
matrix of G + p built from G's matrix must equal solving G + p from scratch,
bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2407_07058_gb300 import appd
from tests.test_gpu_parity import assert_bits, from_dev, to_dev
from tests.test_oracle_pins import sym_random

pytestmark = pytest.mark.gpu


def split(Wf):
    n = Wf.shape[0] - 1
    return np.ascontiguousarray(Wf[:n, :n]), np.ascontiguousarray(Wf[n, :n])


@pytest.mark.parametrize("n", [1, 2, 3, 31, 257, 1000, 1031])
@pytest.mark.parametrize("kind", ["f32", "ties"])
@pytest.mark.parametrize("widest", [False, True])
def test_insert_vertex_parity(n, kind, widest):
    rng = np.random.default_rng(9000 + n)
    Wf = sym_random(n + 1, rng, np.float32) if kind == "f32" else sym_random(n + 1, rng, np.uint32, "ties")
    W, w = split(Wf)
    M = appd.solve(to_dev(W), widest=widest)
    Mo = appd.insert_vertex(M, to_dev(w), widest=widest)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    assert_bits(from_dev(Mo, Wf), oracle.appd(Wf, widest=widest), f"insert n={n} {kind} widest={widest}")


def test_insert_into_empty_graph():
    M = torch.empty((0, 0), dtype=torch.float32, device="cuda")
    Mo = appd.insert_vertex(M, torch.empty(0, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert Mo.shape == (1, 1) and int(Mo.view(torch.int32).item()) == 0


def test_insert_vertex_n16384():
    P = synth.uniform_points(16385, 2, seed=77)
    Wf = synth.euclid(P)
    W, w = split(Wf)
    Mo = appd.insert_vertex(appd.solve(to_dev(W)), to_dev(w))
    torch.cuda.synchronize()
    assert_bits(from_dev(Mo, Wf), oracle.appd(Wf), "insert n=16384")


def test_repeated_insertion_on_device():
    Wf = synth.euclid(synth.gmm_points(200, 2, 3, sigma=0.5, seed=5, mean_box=5.0))
    M = appd.solve(to_dev(np.ascontiguousarray(Wf[:2, :2])))
    for m in range(2, 200):
        M = appd.insert_vertex(M, to_dev(np.ascontiguousarray(Wf[m, :m])))
    torch.cuda.synchronize()
    assert_bits(from_dev(M, Wf), oracle.appd(Wf), "200 insertions")


def test_insert_rejects_overlap():
    M = torch.zeros((10, 10), dtype=torch.float32, device="cuda")
    w = torch.zeros(10, dtype=torch.float32, device="cuda")
    big = torch.zeros(200, dtype=torch.float32, device="cuda")
    lib = appd.load()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.appd_insert_vertex(M.data_ptr(), 10, 0, w.data_ptr(), M.data_ptr(), s) == 8
    assert lib.appd_insert_vertex(M.data_ptr(), 10, 0, big.data_ptr(), big.data_ptr(), s) == 8
