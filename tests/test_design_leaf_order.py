"""CPU check of the leaf-order construction the CUDA dendrogram step uses.

Claim (a restatement of Prim's order on the MST, see Section 3's ascending
form): root the MST at vertex 0; give every non-root vertex y the order value
ord(y) = (weight key of y's parent edge, y); let nha(y) be the nearest proper
ancestor z of parent(y) (walking up, z's own parent edge) with ord(z) > ord(y),
or the root if none.  The preorder of the tree y -> nha(y), children visited in
increasing ord, puts the root first, and the gap between consecutive vertices
x, y of that order is the weight of y's parent edge.  Then
M(i,j) = max of the gaps between pos(i) and pos(j).

This test builds that order in plain Python from the oracle's MST and checks
the range-max reconstruction against the oracle's full matrix.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import keys_np, sym_random


def leaf_order(W):
    n = W.shape[0]
    _, mst = oracle.prim(W)
    K = keys_np(W)
    adj = [[] for _ in range(n)]
    for c in mst.tolist():
        a, b = (c >> 16) & 0xFFFF, c & 0xFFFF
        adj[a].append(b)
        adj[b].append(a)
    parent = [-1] * n
    parent[0] = 0
    stack = [0]
    while stack:
        v = stack.pop()
        for w in adj[v]:
            if parent[w] < 0:
                parent[w] = v
                stack.append(w)
    INF = 1 << 62
    ordv = [INF] * n
    for y in range(1, n):
        p = parent[y]
        ordv[y] = (int(K[min(y, p), max(y, p)]) << 16) | y
    nha = [0] * n
    for y in range(1, n):
        z = parent[y]
        while z != 0 and ordv[z] < ordv[y]:
            z = parent[z]
        nha[y] = z
    kids = [[] for _ in range(n)]
    for y in sorted(range(1, n), key=lambda v: ordv[v]):
        kids[nha[y]].append(y)
    order = []
    stack = [0]
    while stack:
        v = stack.pop()
        order.append(v)
        stack.extend(reversed(kids[v]))
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    gapbits = np.zeros(max(n - 1, 1), dtype=np.uint32)
    gapkey = np.zeros(max(n - 1, 1), dtype=np.uint64)
    for y in range(1, n):
        p = parent[y]
        gapbits[pos[y] - 1] = W.view(np.uint32)[min(y, p), max(y, p)]
        gapkey[pos[y] - 1] = K[min(y, p), max(y, p)]
    return pos, gapbits, gapkey


def rebuild(W):
    n = W.shape[0]
    pos, gb, gk = leaf_order(W)
    M = np.zeros((n, n), dtype=np.uint32)
    for i in range(n):
        for j in range(n):
            if i != j:
                a, b = sorted((pos[i], pos[j]))
                k = int(np.argmax(gk[a:b])) + a
                M[i, j] = gb[k]
    return M.view(W.dtype)


@pytest.mark.parametrize("seed", range(4))
def test_leaf_order_reproduces_oracle(seed):
    rng = np.random.default_rng(100 + seed)
    cases = [sym_random(n, rng, dt, k) for n in (1, 2, 3, 9, 40)
             for dt in (np.float32, np.uint32) for k in ("uniform", "ties")]
    cases.append(synth.euclid(synth.gmm_points(150, 2, 5, sigma=0.5, seed=seed, mean_box=10.0)))
    cases.append(synth.euclid(synth.uniform_points(150, 1, seed=seed)))
    for W in cases:
        ref = oracle.appd(W)
        assert np.array_equal(rebuild(W).view(np.uint32), ref.view(np.uint32))
