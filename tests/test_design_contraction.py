"""The schedule of the bulk-copy level-0 contraction, modelled in plain Python
on CPU and checked against a direct upper-triangle contraction.

The model follows the kernel's decomposition: work items of at most 16 rows of
one group, rows ascending; for every chunk of columns, one stage per row that
reaches the chunk (its segment starts at its first 4-column group right of its
diagonal; groups left of it hold stale data, filled with noise here); running
(key, row) minima per column across the chunk's rows, first strictly smaller
wins; one fold per chunk into bins indexed by the column's group, skipping the
item's own group and columns not right of the item's smallest row.  The
result must equal P(A, B) = min over a in A, b in B, a < b of the packed edge
(key, a, b).  The mbarrier phase arithmetic of the ring (which slot a stage
uses, which parity a wait names) is checked separately.
"""
import numpy as np
import pytest

INF = (1 << 64) - 1
CROWS = 16


def first_group_col(row):
    return ((row + 1) >> 2) << 2


def direct_p(W, lab, cn):
    n = W.shape[0]
    P = [[INF] * cn for _ in range(cn)]
    for a in range(n):
        for b in range(a + 1, n):
            A, B = lab[a], lab[b]
            if A != B:
                P[A][B] = min(P[A][B], (int(W[a, b]) << 32) | (a << 16) | b)
    return P


def modelled_p(W, lab, cn, ch, rng):
    n = W.shape[0]
    P = [[INF] * cn for _ in range(cn)]
    stages = 0
    for A in range(cn):
        members = rng.permutation(np.flatnonzero(lab == A))
        chunks = [members[i:i + CROWS] for i in range(0, len(members), CROWS)]
        for part in chunks:
            rows = sorted(int(r) for r in part)
            r0 = rows[0]
            bins = {}
            c0 = min(first_group_col(r0), n)
            while True:
                c1 = min(n, c0 + ch)
                bk = [0] * (c1 - c0)
                bi = [0] * (c1 - c0)
                for q, row in enumerate(rows):
                    if q > 0 and first_group_col(row) >= c1:
                        break                      # this row and all later ones miss the chunk
                    stages += 1
                    s0 = max(c0, first_group_col(row))
                    seg = rng.integers(0, 2**32, size=c1 - c0)   # stale stage contents
                    seg[s0 - c0:] = W[row, s0:c1]
                    for j in range(c0, c1, 4):
                        for c in range(4):
                            col, k = j + c, int(seg[j + c - c0])
                            if q == 0:
                                bk[col - c0], bi[col - c0] = k, row   # the smallest row seeds
                            elif j + 3 > row and col > row and k < bk[col - c0]:
                                bk[col - c0], bi[col - c0] = k, row
                for col in range(c0, c1):                           # one fold per chunk
                    B = lab[col]
                    if B != A and col > r0:
                        e = (bk[col - c0] << 32) | (bi[col - c0] << 16) | col
                        bins[B] = min(bins.get(B, INF), e)
                if c1 >= n:
                    break
                c0 = c1
            for B, e in bins.items():
                P[A][B] = min(P[A][B], e)
    return P, stages


@pytest.mark.parametrize("n,cn,ch,ties", [(64, 7, 16, False), (100, 30, 8, True), (128, 3, 32, False),
                                          (96, 40, 64, True), (200, 25, 1024, False), (8, 8, 4, False),
                                          (4, 2, 8, True)])
def test_chunked_running_minima_equal_the_direct_contraction(n, cn, ch, ties):
    rng = np.random.default_rng(n * 31 + cn)
    W = rng.integers(0, 8 if ties else 2**31, size=(n, n), dtype=np.uint64)
    W = np.triu(W, 1)
    W = W + W.T
    lab = rng.integers(0, cn, size=n)
    lab[:cn] = np.arange(cn)                 # every group non-empty
    rng.shuffle(lab)
    got, stages = modelled_p(W, lab, cn, ch, rng)
    assert got == direct_p(W, lab, cn)
    assert stages > 0


def test_ring_phase_arithmetic():
    # stage i uses slot i % S and completes phase i // S of that slot's full
    # barrier; a wait for parity p passes once the phase of that parity just
    # before the current one has completed.  After an end marker (stage `it`)
    # the producer may wait only for stages it-S+1 .. it-1: the marker reused
    # the slot of stage it-S, whose phase parity is the slot's current one.
    S = 4
    for it in range(0, 40):
        for end_sent in (False, True):
            used = {}
            for i in range(it + (1 if end_sent else 0)):
                used[i % S] = used.get(i % S, 0) + 1
            lo = (max(0, it + 1 - S) if end_sent else max(0, it - S))
            for i in range(lo, it):
                current = used[i % S]            # index of the slot's incomplete phase
                assert (i // S) & 1 != current & 1
            if end_sent and it >= S:
                i = it - S                       # the reused slot: its wait would never pass
                assert (i // S) & 1 == used[i % S] & 1
