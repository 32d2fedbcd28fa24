"""Pins for the oracle's warm start (Section 6.1): inserting a vertex into a
solved matrix must give what solving the larger graph from scratch gives
(the full solve is pinned in tests/test_oracle_pins.py), bit for bit, for
both dtypes, with ties and special values, and for widest paths."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import sym_random


def split(Wfull: np.ndarray):
    n = Wfull.shape[0] - 1
    return np.ascontiguousarray(Wfull[:n, :n]), np.ascontiguousarray(Wfull[n, :n])


@pytest.mark.parametrize("n", [1, 2, 3, 7, 40, 301])
@pytest.mark.parametrize("kind", ["f32", "u32", "ties"])
@pytest.mark.parametrize("widest", [False, True])
def test_insert_equals_solving_from_scratch(n, kind, widest):
    rng = np.random.default_rng(100 * n + len(kind))
    if kind == "f32":
        Wf = sym_random(n + 1, rng, np.float32)
    elif kind == "u32":
        Wf = sym_random(n + 1, rng, np.uint32)
    else:
        Wf = sym_random(n + 1, rng, np.uint32, "ties")
    W, w = split(Wf)
    got = oracle.insert(oracle.appd(W, widest=widest), w, widest=widest)
    assert np.array_equal(got.view(np.uint32), oracle.appd(Wf, widest=widest).view(np.uint32))


def test_repeated_insertion_builds_the_whole_matrix():
    Wf = synth.euclid(synth.gmm_points(60, 2, 3, sigma=0.5, seed=9, mean_box=5.0))
    M = oracle.appd(np.ascontiguousarray(Wf[:2, :2]))
    for m in range(2, 60):
        M = oracle.insert(M, np.ascontiguousarray(Wf[m, :m]))
    assert np.array_equal(M.view(np.uint32), oracle.appd(Wf).view(np.uint32))


def test_insert_planted_mistake_is_caught():
    # dropping the path through the new vertex (M' = M off the new row) fails
    rng = np.random.default_rng(3)
    Wf = sym_random(30, rng, np.float32)
    W, w = split(Wf)
    M = oracle.appd(W)
    wrong = np.zeros((30, 30), np.float32)
    wrong[:29, :29] = M
    ref = oracle.appd(Wf)
    assert not np.array_equal(wrong[:29, :29].view(np.uint32), ref[:29, :29].view(np.uint32))
    assert np.array_equal(oracle.insert(M, w).view(np.uint32), ref.view(np.uint32))
