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


# ---------------------------------------------- warm start through the tree
def _tree_triples(keys, lo, hi):
    t = np.stack([keys.cpu().numpy().view(np.uint32), lo.cpu().numpy().view(np.uint32),
                  hi.cpu().numpy().view(np.uint32)], axis=1).astype(np.uint64)
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]


def _oracle_triples(W, widest=False):
    n = W.shape[0]
    _, mst = oracle.prim(W, widest=widest)
    lo, hi = oracle.code_ends(mst, n)
    t = np.stack([mst >> 32, lo, hi], axis=1).astype(np.uint64)
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]


@pytest.mark.parametrize("n", [1, 2, 3, 31, 257, 1000, 4099, 8191, 8192, 9000])
@pytest.mark.parametrize("kind", ["f32", "ties"])
@pytest.mark.parametrize("widest", [False, True])
def test_insert_vertex_tree_parity(n, kind, widest):
    """G's tree (mst_edges) and p's weights give G + p's matrix and tree: the
    matrix equals the oracle's solve of G + p, the tree its Prim tree."""
    rng = np.random.default_rng(9500 + n)
    Wf = sym_random(n + 1, rng, np.float32) if kind == "f32" else sym_random(n + 1, rng, np.uint32, "ties")
    W, w = split(Wf)
    T = to_dev(W)
    tree = appd.mst_edges(T, widest=widest)
    Mo, nt = appd.insert_vertex_tree(tree, to_dev(w), n, T.dtype, widest=widest)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    assert_bits(from_dev(Mo, Wf), oracle.appd(Wf, widest=widest), f"tree insert n={n} {kind}")
    assert np.array_equal(_tree_triples(*nt), _oracle_triples(Wf, widest)), "new tree differs"


def test_insert_vertex_tree_chained():
    """120 vertices inserted one after another, each call given the tree the
    previous one returned: the last matrix equals solving the whole graph."""
    Wf = synth.euclid(synth.gmm_points(1120, 2, 4, sigma=0.5, seed=8, mean_box=6.0))
    n0 = 1000
    tree = appd.mst_edges(to_dev(np.ascontiguousarray(Wf[:n0, :n0])))
    for m in range(n0, 1120):
        Mo, tree = appd.insert_vertex_tree(tree, to_dev(np.ascontiguousarray(Wf[m, :m])), m, torch.float32)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    assert_bits(from_dev(Mo, Wf), oracle.appd(Wf), "120 chained insertions")


def test_insert_vertex_tree_into_n65536_every_row():
    """The n = 65536 mixture graph plus one vertex: the new tree has 65537
    vertices (pair numbers past 16 bits); every row is checked against the
    oracle on the extended graph."""
    n = 65536
    pts = synth.cfg3_points(n + 1)
    st = torch.cuda.current_stream().cuda_stream
    Pd = torch.from_numpy(pts).cuda()
    Wf = torch.empty((n + 1, n + 1), dtype=torch.float32, device="cuda")
    synth.device_euclid(Pd.data_ptr(), n + 1, 16, Wf.data_ptr(), st)
    W = Wf[:n, :n].contiguous()
    w = Wf[n, :n].contiguous()
    tree = appd.mst_edges(W)
    del W
    Mo, _ = appd.insert_vertex_tree(tree, w, n, torch.float32, tree_out=False)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    Wh = Wf.cpu().numpy()
    del Wf
    order, mst = oracle.prim_sym(Wh)   # W is symmetric by construction
    for r0 in range(0, n + 1, 4096):
        r1 = min(n + 1, r0 + 4096)
        ref = oracle.prim_rows(Wh, order, mst, np.arange(r0, r1))
        assert_bits(Mo[r0:r1].cpu().numpy(), ref, f"insert into n={n}, rows {r0}..")


def test_insert_vertex_tree_arguments():
    lib = appd.load()
    s = torch.cuda.current_stream().cuda_stream
    M = torch.zeros((11, 11), dtype=torch.float32, device="cuda")
    t = torch.zeros(9, dtype=torch.int32, device="cuda")
    w = torch.zeros(10, dtype=torch.float32, device="cuda")
    p = t.data_ptr()
    assert lib.appd_insert_vertex_tree(None, p, p, 10, 0, w.data_ptr(), M.data_ptr(), None, None, None, s) == 1
    assert lib.appd_insert_vertex_tree(p, p, p, 10, 0, M.data_ptr(), M.data_ptr(), None, None, None, s) == 8
    assert lib.appd_insert_vertex_tree(p, p, p, 92682, 0, w.data_ptr(), M.data_ptr(), None, None, None, s) == 2
    z = torch.full((1, 1), 7, dtype=torch.int32, device="cuda")
    assert lib.appd_insert_vertex_tree(None, None, None, 0, 1, None, z.data_ptr(), None, None, None, s) == 0
    torch.cuda.synchronize()
    assert int(z.item()) == 0
