"""Pins for the CPU oracle (no GPU).

The oracle (Prim + Algorithm 4, Sections 3 and 5) is checked against things
that do not share its code or its algorithm:

- hand-worked examples in tests/golden/ (Eq. 1-2 applied by hand);
- a Python enumeration of every simple path (Eq. 1-2 written out again);
- threshold connectivity: M(i,j) is the smallest weight t such that i and j
  are connected by edges of weight <= t (an equivalent characterisation of
  the minimax distance, computed with scipy's connected components);
- closed forms: points on a line, all-equal weights, n = 1 and n = 2, two
  well-separated clusters;
- invariants from the proof in Section 5 and from ultrametricity;
- the planted-mistake test: each mutation of the oracle is caught.
"""
import itertools
import struct

import numpy as np
import pytest
from scipy.sparse.csgraph import connected_components

import oracle
import synth
from tests import golden_io


# ------------------------------------------------------------------ helpers
def f32_bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def keys_np(A: np.ndarray) -> np.ndarray:
    """Order keys of a float32/uint32 array (pinned by test_order_key_total_order)."""
    b = A.view(np.uint32).astype(np.uint64)
    if A.dtype == np.uint32:
        return b
    neg = (b >> 31) == 1
    return np.where(neg, (~b) & 0xFFFFFFFF, b | 0x80000000)


def py_brute(W: np.ndarray) -> np.ndarray:
    """Every simple path, Eq. 1-2, in plain Python (n <= 7)."""
    n = W.shape[0]
    K = keys_np(W)
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
                    mk = max(K[path[t], path[t + 1]] for t in range(len(path) - 1))
                    if best is None or mk < best:
                        best = mk
                        arg = max(range(len(path) - 1), key=lambda t: K[path[t], path[t + 1]])
                        bi, bj = path[arg], path[arg + 1]
            out[i, j] = W[bi, bj]
    return out


def threshold_connectivity(W: np.ndarray) -> np.ndarray:
    """M(i,j) = smallest key t with i~j in the graph of edges with key <= t."""
    n = W.shape[0]
    K = keys_np(W)
    off = ~np.eye(n, dtype=bool)
    levels = np.unique(K[off])
    res = np.full((n, n), -1, dtype=np.int64)
    for t in levels:
        adj = (K <= t) & off
        _, lab = connected_components(adj.astype(np.int8), directed=False)
        same = lab[:, None] == lab[None, :]
        newly = same & (res < 0) & off
        res[newly] = t
    # map keys back to bits: take any edge with that key
    out = np.zeros_like(W)
    flatk, flatw = K[off], W.view(np.uint32)[off]
    lut = dict(zip(flatk.tolist(), flatw.tolist()))
    ob = out.view(np.uint32)
    for i in range(n):
        for j in range(n):
            if i != j:
                ob[i, j] = lut[int(res[i, j])]
    return out


def sym_random(n, rng, dtype, kind="uniform"):
    if dtype == np.uint32:
        hi = 3 if kind == "ties" else 1 << 16
        A = rng.integers(0, hi, size=(n, n)).astype(np.uint32)
    else:
        if kind == "ties":
            A = rng.integers(0, 3, size=(n, n)).astype(np.float32)
        else:
            A = rng.random((n, n)).astype(np.float32)
    A = np.triu(A, 1)
    A = A + A.T
    np.fill_diagonal(A, 0)
    return np.ascontiguousarray(A.astype(dtype))


def bits_equal(A, B):
    return np.array_equal(A.view(np.uint32), B.view(np.uint32))


# -------------------------------------------------------------------- tests
def test_order_key_total_order():
    # IEEE-754 totalOrder, listed by hand: -NaN < -inf < -max < -1 < -min_sub
    # < -0 < +0 < +min_sub < 1 < max < +inf < +NaN
    vals = [0xFFC00000, 0xFF800000, 0xFF7FFFFF, 0xBF800000, 0x80000001, 0x80000000,
            0x00000000, 0x00000001, 0x3F800000, 0x7F7FFFFF, 0x7F800000, 0x7FC00000]
    ks = [oracle.order_key(v, oracle.F32) for v in vals]
    assert ks == sorted(ks) and len(set(ks)) == len(ks)
    kn = keys_np(np.array(vals, dtype=np.uint32).view(np.float32)).tolist()
    assert kn == ks
    for v in [0, 1, 77, 0xFFFF, 0xFFFFFFFF]:
        assert oracle.order_key(v, oracle.U32) == v


@pytest.mark.parametrize("path", golden_io.all_fixtures(), ids=lambda p: p.split("/")[-1])
def test_golden_fixtures(path):
    W, M = golden_io.load(path)
    for fn in (oracle.appd, oracle.appd_ascending, oracle.fw, oracle.brute):
        got = fn(W)
        assert bits_equal(got, M), (fn.__name__, got, M)


@pytest.mark.parametrize("dtype", [np.float32, np.uint32])
@pytest.mark.parametrize("kind", ["uniform", "ties"])
def test_small_vs_python_enumeration(dtype, kind):
    rng = np.random.default_rng(11)
    for n in range(1, 7):
        for _ in range(6):
            W = sym_random(n, rng, dtype, kind)
            ref = py_brute(W)
            assert bits_equal(oracle.appd(W), ref)
            assert bits_equal(oracle.brute(W), ref)


@pytest.mark.parametrize("dtype", [np.float32, np.uint32])
@pytest.mark.parametrize("kind", ["uniform", "ties"])
def test_vs_threshold_connectivity(dtype, kind):
    rng = np.random.default_rng(12)
    for n in (7, 8, 9, 23, 47):
        W = sym_random(n, rng, dtype, kind)
        ref = threshold_connectivity(W)
        assert bits_equal(oracle.appd(W), ref)
        if n <= 9:
            assert bits_equal(oracle.brute(W), ref)


def test_fw_and_ascending_agree():
    rng = np.random.default_rng(13)
    cases = [sym_random(n, rng, dt, k) for n in (2, 3, 17, 64, 200)
             for dt in (np.float32, np.uint32) for k in ("uniform", "ties")]
    cases.append(synth.euclid(synth.gmm_points(256, 2, 5, sigma=0.5, seed=9, mean_box=10.0)))
    cases.append(synth.hash_u32(300, seed=7))
    for W in cases:
        A = oracle.appd(W)
        assert bits_equal(A, oracle.fw(W))
        assert bits_equal(A, oracle.appd_ascending(W))


def test_closed_form_points_on_a_line():
    # 1-D Euclidean distances: M(i,j) is the largest gap between consecutive
    # sorted coordinates between x_i and x_j (every path must cross each gap).
    rng = np.random.default_rng(14)
    x = (rng.random(150) * 100).astype(np.float32)
    W = synth.euclid(x[:, None])
    srt = np.argsort(x, kind="stable")
    xs = x[srt].astype(np.float64)
    gaps = np.abs(xs[1:] - xs[:-1]).astype(np.float32)  # |a-b| rounded once to f32
    rank = np.empty(len(x), dtype=np.int64)
    rank[srt] = np.arange(len(x))
    n = len(x)
    ref = np.zeros((n, n), dtype=np.float32)
    for i in range(n):
        for j in range(n):
            if i != j:
                a, b = sorted((rank[i], rank[j]))
                ref[i, j] = gaps[a:b].max()
    assert bits_equal(oracle.appd(W), ref)


def test_closed_forms_degenerate():
    assert bits_equal(oracle.appd(np.zeros((1, 1), np.float32)), np.zeros((1, 1), np.float32))
    W2 = np.array([[0, 2.5], [2.5, 0]], dtype=np.float32)
    assert bits_equal(oracle.appd(W2), W2)
    n = 40
    E = np.full((n, n), 7, dtype=np.uint32)
    np.fill_diagonal(E, 0)
    assert np.array_equal(oracle.appd(E), E)


def test_two_separated_clusters():
    # Two clusters far apart: every cross pair equals the smallest
    # inter-cluster distance; within a cluster the answer is the cluster's own.
    rng = np.random.default_rng(15)
    a = rng.random((60, 2)).astype(np.float32)
    b = (rng.random((50, 2)) + 100.0).astype(np.float32)
    pts = np.vstack([a, b])
    W = synth.euclid(pts)
    M = oracle.appd(W)
    cross = W[:60, 60:].min()
    assert np.all(M[:60, 60:] == cross) and np.all(M[60:, :60] == cross)
    assert bits_equal(M[:60, :60], oracle.appd(np.ascontiguousarray(W[:60, :60])))
    assert bits_equal(M[60:, 60:], oracle.appd(np.ascontiguousarray(W[60:, 60:])))


@pytest.mark.parametrize("which", ["gmm", "u32", "uniform01"])
def test_invariants(which):
    if which == "gmm":
        W = synth.euclid(synth.gmm_points(120, 2, 5, sigma=0.5, seed=3, mean_box=10.0))
    elif which == "u32":
        W = synth.hash_u32(120, seed=5)
    else:
        W = synth.uniform01(120, seed=6)
    n = W.shape[0]
    M, cnt = oracle.appd(W, return_fill_count=True)
    assert cnt == n * (n - 1)                       # each off-diagonal cell once
    assert bits_equal(M, np.ascontiguousarray(M.T))  # symmetry
    assert np.all(M.view(np.uint32).diagonal() == 0)
    order, mst = oracle.prim(W)
    lo = ((mst >> 16) & 0xFFFF).astype(np.int64)
    hi = (mst & 0xFFFF).astype(np.int64)
    mst_bits = set(W.view(np.uint32)[lo, hi].tolist())
    off = ~np.eye(n, dtype=bool)
    assert set(M.view(np.uint32)[off].tolist()) <= mst_bits  # every value is an MST weight
    assert bits_equal(M[lo, hi], W[lo, hi])                 # MST edges are their own answer
    KM, KW = keys_np(M), keys_np(W)
    assert np.all(KM[off] <= KW[off])                        # M <= W
    # ultrametric: M(i,k) <= max(M(i,j), M(j,k)) for all triples
    lhs = KM[:, None, :]
    rhs = np.maximum(KM[:, :, None], KM[None, :, :])
    assert np.all(lhs <= rhs)
    # histogram: each MST edge accounts for |tree1|*|tree2| pairs (Section 5),
    # checked here as: count of pairs at each value == sum over MST edges of
    # that weight of the product of the two side sizes when removed.
    adj = {v: [] for v in range(n)}
    for a, b in zip(lo.tolist(), hi.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    from collections import Counter
    want = Counter()
    for a, b, bits in zip(lo.tolist(), hi.tolist(), W.view(np.uint32)[lo, hi].tolist()):
        # side of a after removing a-b, restricted to edges with larger-or-equal
        # position in the strict order is not needed: Section 5 counts pairs
        # whose tree path maximum is this edge.
        code = (int(KW[a, b]) << 32) | (a << 16) | b
        stack, seen = [a], {a}
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if w in seen or {v, w} == {a, b}:
                    continue
                c = (int(KW[min(v, w), max(v, w)]) << 32) | (min(v, w) << 16) | max(v, w)
                if c < code:
                    seen.add(w)
                    stack.append(w)
        s1 = len(seen)
        stack, seen2 = [b], {b}
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if w in seen2 or {v, w} == {a, b}:
                    continue
                c = (int(KW[min(v, w), max(v, w)]) << 32) | (min(v, w) << 16) | max(v, w)
                if c < code:
                    seen2.add(w)
                    stack.append(w)
        want[bits] += 2 * s1 * len(seen2)
    have = Counter(M.view(np.uint32)[off].tolist())
    assert have == want
    assert sum(want.values()) == n * (n - 1)


def test_prim_order_identity():
    # With Prim's order v_0..v_{n-1} and delta_k the weight that added v_k,
    # M(v_a, v_b) = max_{a<k<=b} delta_k.  An independent second route to M.
    for W in (synth.euclid(synth.uniform_points(300, 2, seed=21)), synth.hash_u32(257, seed=22)):
        M = oracle.appd(W)
        order, mst = oracle.prim(W)
        n = W.shape[0]
        dk = (mst >> 32).astype(np.uint64)
        lo = ((mst >> 16) & 0xFFFF).astype(np.int64)
        hi = (mst & 0xFFFF).astype(np.int64)
        dbits = W.view(np.uint32)[lo, hi]
        ref = np.zeros((n, n), dtype=np.uint32)
        for a in range(n):
            best_k, best_b = 0, 0
            for b in range(a + 1, n):
                if b == a + 1 or dk[b - 1] > best_k:
                    best_k, best_b = dk[b - 1], dbits[b - 1]
                ref[order[a], order[b]] = best_b
                ref[order[b], order[a]] = best_b
        assert np.array_equal(M.view(np.uint32), ref)


def test_tree_rows_match_full_matrix():
    W = synth.euclid(synth.gmm_points(400, 16, 8, sigma=1.0, seed=23, mean_std=5.0))
    M = oracle.appd(W)
    _, mst = oracle.prim(W)
    src = [0, 5, 199, 399]
    rows = oracle.tree_rows(W, mst, src)
    assert bits_equal(rows, np.ascontiguousarray(M[src]))


def test_special_values():
    # NaN, infinities, signed zeros and negatives compare by totalOrder; the
    # output keeps each selected weight's own bits.
    rng = np.random.default_rng(24)
    pool = np.array([0xFFC00000, 0xFF800000, 0xBF800000, 0x80000000, 0x00000000, 0x3F800000,
                     0x7F800000, 0x7FC00000, 0x40000000, 0x7FC00001], dtype=np.uint32)
    for n in (3, 5, 6):
        for _ in range(5):
            B = pool[rng.integers(0, len(pool), size=(n, n))]
            B = np.triu(B, 1)
            B = B + B.T
            np.fill_diagonal(B, 0)
            W = np.ascontiguousarray(B.astype(np.uint32)).view(np.float32)
            ref = py_brute(W)
            assert bits_equal(oracle.appd(W), ref)
            assert bits_equal(oracle.fw(W), ref)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(k):
    rng = np.random.default_rng(25)
    Ws = [sym_random(6, rng, np.float32, "uniform"), sym_random(30, rng, np.uint32, "uniform"),
          synth.euclid(synth.uniform_points(40, 2, seed=26))]
    refs = [threshold_connectivity(W) for W in Ws]
    caught = False
    with oracle.mutation(k):
        for W, ref in zip(Ws, refs):
            M, cnt = oracle.appd(W, return_fill_count=True)
            n = W.shape[0]
            if not bits_equal(M, ref) or cnt != n * (n - 1):
                caught = True
    assert caught, f"mutation {k} not caught by the pins"
    # and the oracle is correct again afterwards
    assert bits_equal(oracle.appd(Ws[0]), refs[0])


# ------------------------------------------------ rows from Prim's order
@pytest.mark.parametrize("widest", [False, True])
def test_prim_rows_equal_full_matrix(widest):
    # every row read off Prim's visiting order equals the Algorithm 4 matrix,
    # on ties, special values and both dtypes
    rng = np.random.default_rng(31)
    cases = [synth.euclid(synth.uniform_points(300, 2, seed=32)), synth.hash_u32(257, seed=33),
             sym_random(64, rng, np.uint32, "ties"), sym_random(50, rng, np.float32, "ties"),
             sym_random(2, rng, np.float32), sym_random(1, rng, np.uint32)]
    pool = np.array([0xFFC00000, 0xFF800000, 0xBF800000, 0x80000000, 0x00000000, 0x3F800000,
                     0x7F800000, 0x7FC00000], dtype=np.uint32)
    B = np.triu(pool[rng.integers(0, len(pool), size=(40, 40))], 1)
    B = B + B.T
    np.fill_diagonal(B, 0)
    cases.append(np.ascontiguousarray(B.astype(np.uint32)).view(np.float32))
    for W in cases:
        n = W.shape[0]
        order, mst = oracle.prim(W, widest=widest)
        rows = oracle.prim_rows(W, order, mst, np.arange(n), widest=widest)
        assert bits_equal(rows, oracle.appd(W, widest=widest)), f"n={n}"


def test_prim_rows_vs_threshold_connectivity():
    rng = np.random.default_rng(34)
    for W in (sym_random(12, rng, np.uint32, "ties"), sym_random(15, rng, np.float32)):
        order, mst = oracle.prim(W)
        rows = oracle.prim_rows(W, order, mst, np.arange(W.shape[0]))
        assert bits_equal(rows, threshold_connectivity(W))


def test_prim_rows_planted_mistake_is_caught():
    W = synth.euclid(synth.uniform_points(60, 2, seed=35))
    order, mst = oracle.prim(W)
    ref = threshold_connectivity(W)
    with oracle.mutation(5):
        bad = oracle.prim_rows(W, order, mst, np.arange(60))
    assert not bits_equal(bad, ref)
    assert bits_equal(oracle.prim_rows(W, order, mst, np.arange(60)), ref)


# ----------------------------------------- FP32 weights of a point set
def _round_f32(x) -> np.float32:
    """Round an exact rational to the nearest FP32 value, ties to even."""
    from fractions import Fraction
    x = Fraction(x)
    if x == 0:
        return np.float32(0.0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)                       # subnormals share the smallest exponent
    scale = Fraction(2) ** (23 - e)
    m = a * scale
    q, r = divmod(m.numerator, m.denominator)
    twice = 2 * r
    if twice > m.denominator or (twice == m.denominator and q % 2 == 1):
        q += 1
    return np.float32(sign * float(Fraction(q) / scale))


def _sqrt_f32(s: np.float32) -> np.float32:
    """Correctly rounded FP32 square root, decided with exact rationals."""
    import math
    from fractions import Fraction
    if s == 0:
        return np.float32(0.0)
    S = Fraction(float(s))
    r = np.float32(math.sqrt(float(s)))
    for c in (np.nextafter(r, np.float32(0)), r, np.nextafter(r, np.float32(np.inf))):
        lo = (Fraction(float(np.nextafter(c, np.float32(0)))) + Fraction(float(c))) / 2
        hi = (Fraction(float(c)) + Fraction(float(np.nextafter(c, np.float32(np.inf))))) / 2
        if lo * lo <= S <= hi * hi:
            return c
    raise AssertionError("no correctly rounded candidate")


def _points_w_exact(X: np.ndarray) -> np.ndarray:
    """Each step of the definition with exact rationals and one rounding."""
    from fractions import Fraction
    n, d = X.shape
    W = np.zeros((n, n), dtype=np.float32)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            s = np.float32(0.0)
            for k in range(d):
                t = _round_f32(Fraction(float(X[i, k])) - Fraction(float(X[j, k])))
                s = _round_f32(Fraction(float(t)) * Fraction(float(t)) + Fraction(float(s)))
            W[i, j] = _sqrt_f32(s)
    return W


def test_points_w_vs_exact_rational_steps():
    for X in (synth.gmm_points(9, 16, 3, sigma=1.0, seed=36, mean_std=5.0),
              synth.uniform_points(12, 2, seed=37),
              synth.gmm_points(7, 3, 2, sigma=1e-3, seed=38, mean_box=1e4)):
        assert bits_equal(oracle.points_w(X), _points_w_exact(X))


def test_points_w_vs_numpy_where_products_are_exact():
    # coordinates on a grid of 2^-6 with small integer parts: every difference
    # has at most 12 significant bits, so t*t is exact in FP32 and the fused
    # step equals numpy's float32 multiply then add in the same order
    rng = np.random.default_rng(39)
    X = (rng.integers(-2000, 2000, size=(40, 5)) / 64.0).astype(np.float32)
    n, d = X.shape
    ref = np.zeros((n, n), dtype=np.float32)
    for i in range(n):
        s = np.zeros(n, dtype=np.float32)
        for k in range(d):
            t = (X[i, k] - X[:, k]).astype(np.float32)
            s = (s + (t * t).astype(np.float32)).astype(np.float32)
        ref[i] = np.sqrt(s).astype(np.float32)
    np.fill_diagonal(ref, 0)
    assert bits_equal(oracle.points_w(X), ref)


def test_points_w_vs_fp64_generator_on_integer_points():
    # integer coordinates: every step is exact in both, so the FP32 definition
    # and the FP64-then-rounded generator agree
    rng = np.random.default_rng(40)
    X = rng.integers(-300, 300, size=(64, 16)).astype(np.float32)
    W = oracle.points_w(X)
    assert bits_equal(W, synth.euclid(X))
    assert bits_equal(W, np.ascontiguousarray(W.T))
    assert not np.any(np.diag(W).view(np.uint32))


# ------------------------------- pair numbers of graphs above 65536 vertices
def test_rank_pair_numbers_on_small_graphs():
    # Graphs above 65536 vertices number a pair by its rank among all pairs in
    # (lo, hi) order.  Forced onto small graphs, every routine that uses edge
    # codes must still give the pinned matrix, and the codes must rank the
    # pairs: code_ends inverts them and they sort as (key, lo, hi).
    rng = np.random.default_rng(41)
    cases = [sym_random(7, rng, np.float32), sym_random(40, rng, np.uint32, "ties"),
             synth.euclid(synth.uniform_points(200, 2, seed=42)), synth.hash_u32(2, seed=43)]
    refs = [threshold_connectivity(W) if W.shape[0] <= 40 else oracle.fw(W) for W in cases]
    with oracle.short_limit(1):
        for W, ref in zip(cases, refs):
            n = W.shape[0]
            assert bits_equal(oracle.appd(W), ref)
            assert bits_equal(oracle.appd_ascending(W), ref)
            order, mst = oracle.prim(W)
            assert bits_equal(oracle.prim_rows(W, order, mst, np.arange(n)), ref)
            assert bits_equal(oracle.tree_rows(W, mst, np.arange(n)), ref)
            lo, hi = oracle.code_ends(mst, n)
            assert np.all(lo < hi) and np.all(hi < n)
            rank = lo.astype(np.int64) * (n - 1) - lo.astype(np.int64) * (lo.astype(np.int64) - 1) // 2 \
                + (hi.astype(np.int64) - lo.astype(np.int64) - 1)
            assert np.array_equal(mst & 0xFFFFFFFF, rank.astype(np.uint64))
            K = keys_np(W)
            assert np.array_equal(mst >> 32, K[lo, hi])
        # every pair of a 300-vertex graph: the rank is a bijection onto
        # 0 .. n(n-1)/2 - 1 that code_ends inverts
        n = 300
        ii, jj = np.triu_indices(n, 1)
        r = (ii * (n - 1) - ii * (ii - 1) // 2 + (jj - ii - 1)).astype(np.uint64)
        assert np.array_equal(np.sort(r), np.arange(n * (n - 1) // 2, dtype=np.uint64))
        lo, hi = oracle.code_ends(r, n)
        assert np.array_equal(lo, ii.astype(np.uint32)) and np.array_equal(hi, jj.astype(np.uint32))
    # and the short form is back
    order, mst = oracle.prim(cases[1])
    assert np.array_equal((mst >> 16) & 0xFFFF, oracle.code_ends(mst, 40)[0])


def test_prim_sym_equals_prim_on_symmetric_input():
    rng = np.random.default_rng(44)
    cases = [synth.euclid(synth.uniform_points(500, 2, seed=45)), synth.hash_u32(300, seed=46),
             sym_random(64, rng, np.uint32, "ties"), sym_random(2, rng, np.float32)]
    for W in cases:
        for widest in (False, True):
            o1, m1 = oracle.prim(W, widest=widest)
            o2, m2 = oracle.prim_sym(W, widest=widest)
            assert np.array_equal(o1, o2) and np.array_equal(m1, m2)
        with oracle.short_limit(1):
            o1, m1 = oracle.prim(W)
            o2, m2 = oracle.prim_sym(W)
            assert np.array_equal(o1, o2) and np.array_equal(m1, m2)
