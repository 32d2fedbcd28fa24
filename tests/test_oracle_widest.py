"""Pins for the oracle's widest-path matrix (Section 4.2), no GPU.

The widest-path distance of i and j is the largest possible smallest edge
weight over all i-j paths.  The oracle computes it with the same routines as
the minimax matrix and the order of every comparison reversed (a maximum
spanning tree whose edges are removed in ascending order).  Pinned here
against things that share none of that code:

- every simple path enumerated in plain Python with the weights' own numeric
  order (no order keys);
- threshold connectivity: the largest weight t such that i and j are
  connected by edges of weight >= t (scipy's connected components);
- duality with the pinned minimax oracle: negating a float flips its
  totalOrder, so off the diagonal widest(W) = -minimax(-W) bit for bit;
- the maximum spanning tree's total weight against scipy's minimum spanning
  tree of the negated weights;
- invariants, and the planted mistakes of the oracle.
"""
import itertools

import numpy as np
import pytest
from scipy.sparse.csgraph import connected_components, minimum_spanning_tree

import oracle
import synth


def sym_from(upper: np.ndarray, dtype) -> np.ndarray:
    A = np.triu(upper, 1)
    A = A + A.T
    np.fill_diagonal(A, 0)
    return np.ascontiguousarray(A.astype(dtype))


def rand_f32(n, seed, lo=0.5, hi=9.5):
    rng = np.random.default_rng(seed)
    return sym_from(rng.uniform(lo, hi, (n, n)), np.float32)


def rand_u32(n, seed, top=12):
    rng = np.random.default_rng(seed)
    return sym_from(rng.integers(1, top, (n, n)), np.uint32)


def py_widest(W: np.ndarray) -> np.ndarray:
    """Every simple path, numeric order of the weights (finite, no zeros)."""
    n = W.shape[0]
    out = np.zeros_like(W)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            best = None
            others = [v for v in range(n) if v not in (i, j)]
            for r in range(len(others) + 1):
                for mid in itertools.permutations(others, r):
                    path = (i,) + mid + (j,)
                    m = min(W[path[t], path[t + 1]] for t in range(len(path) - 1))
                    if best is None or m > best:
                        best = m
            out[i, j] = best
    return out


def threshold_widest(W: np.ndarray) -> np.ndarray:
    """Largest t with i, j connected by edges of weight >= t."""
    n = W.shape[0]
    off = ~np.eye(n, dtype=bool)
    out = np.zeros_like(W)
    done = np.eye(n, dtype=bool)
    for t in sorted(set(W[off].tolist()), reverse=True):
        adj = (W >= t) & off
        _, lab = connected_components(adj.astype(np.int8), directed=False)
        same = lab[:, None] == lab[None, :]
        new = same & ~done
        out[new] = t
        done |= same
    return out


@pytest.mark.parametrize("n,seed", [(4, 1), (5, 2), (6, 3), (7, 4)])
def test_widest_equals_path_enumeration(n, seed):
    for W in (rand_f32(n, seed), rand_u32(n, seed + 50)):
        assert np.array_equal(oracle.appd(W, widest=True), py_widest(W))
        assert np.array_equal(oracle.brute(W, widest=True), py_widest(W))


@pytest.mark.parametrize("n,seed", [(12, 5), (30, 6), (40, 7)])
def test_widest_equals_threshold_connectivity(n, seed):
    for W in (rand_f32(n, seed), rand_u32(n, seed + 50, top=6)):
        assert np.array_equal(oracle.appd(W, widest=True), threshold_widest(W))


def flip(W: np.ndarray) -> np.ndarray:
    return (W.view(np.uint32) ^ np.uint32(0x80000000)).view(np.float32)


@pytest.mark.parametrize("seed", [8, 9])
def test_widest_is_negated_minimax_of_negated_weights(seed):
    n = 60
    rng = np.random.default_rng(seed)
    W = sym_from(rng.normal(0, 3, (n, n)), np.float32)
    # special values too: the sign flip reverses totalOrder exactly
    pool = np.array([np.inf, -np.inf, 0.0, -0.0, np.nan, 1.0, -1.0], np.float32)
    idx = rng.integers(0, n, (40, 2))
    for a, b in idx:
        if a != b:
            W[a, b] = W[b, a] = pool[rng.integers(0, len(pool))]
    got = oracle.appd(W, widest=True).view(np.uint32)
    ref = flip(oracle.appd(flip(W))).view(np.uint32)
    off = ~np.eye(n, dtype=bool)
    assert np.array_equal(got[off], ref[off])
    assert not got[~off].any()


def test_maximum_spanning_tree_weight():
    n = 50
    W = rand_f32(n, 10)
    _, codes = oracle.prim(W, widest=True)
    lo = (codes >> 16) & 0xFFFF
    hi = codes & 0xFFFF
    total = float(np.sum(W[lo.astype(int), hi.astype(int)].astype(np.float64)))
    ref = -minimum_spanning_tree(-W.astype(np.float64)).sum()
    assert len(codes) == n - 1
    assert abs(total - ref) < 1e-9 * abs(ref)


def test_widest_routines_agree_and_invariants():
    for W in (rand_f32(80, 11), rand_u32(80, 12, top=20), synth.hash_u32(64, seed=13)):
        M = oracle.appd(W, widest=True)
        assert np.array_equal(M, oracle.appd_ascending(W, widest=True))
        assert np.array_equal(M, oracle.fw(W, widest=True))
        n = W.shape[0]
        off = ~np.eye(n, dtype=bool)
        assert np.array_equal(M, M.T)
        assert not M.view(np.uint32)[~off].any()
        Mv, Wv = M.astype(np.float64), W.astype(np.float64)
        assert (Mv[off] >= Wv[off]).all()                       # the edge itself is a path
        # M(i,k) >= min(M(i,j), M(j,k)) on all triples
        for j in range(n):
            lower = np.minimum(Mv[:, j][:, None], Mv[j, :][None, :])
            assert (Mv[off] >= lower[off]).all()
        # sampled rows by traversing the maximum spanning tree
        _, codes = oracle.prim(W, widest=True)
        rows = oracle.tree_rows(W, codes, [0, 5, n - 1], widest=True)
        assert np.array_equal(rows, M[[0, 5, n - 1]])


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_planted_mistakes_fail_a_widest_pin(k):
    W = rand_f32(7, 14)
    ref = py_widest(W)
    with oracle.mutation(k):
        got = oracle.appd(W, widest=True)
    assert not np.array_equal(got, ref)
