"""Pins of the oracle's similarity-graph functions (Sec. 2.1 graph G_S, Sec. 2.2 k-nn on
the graph) to a hand-worked example, to scipy.sparse, and to a heap-based selection."""
import heapq

import numpy as np
import pytest

import oracle
import synth


def test_hand_worked_graph():
    # matches of a 5-vector set: (0,1) .9, (0,3) .8, (2,3) .95, (1,3) .8; vertex 4 isolated
    i = np.array([0, 0, 1, 2])
    j = np.array([1, 3, 3, 3])
    s = np.array([0.9, 0.8, 0.8, 0.95], dtype=np.float32)
    rp, col, w = oracle.graph_csr(i, j, s, 5)
    assert rp.tolist() == [0, 2, 4, 5, 8, 8]
    assert col.tolist() == [1, 3, 0, 3, 3, 0, 1, 2]
    assert np.allclose(w, [0.9, 0.8, 0.9, 0.8, 0.95, 0.8, 0.8, 0.95])
    nbr, wk = oracle.graph_knn(rp, col, w, 2)
    # vertex 3: weights .8 (0), .8 (1), .95 (2) -> 2 first, then the tie at .8 goes to id 0
    assert nbr.tolist() == [[1, 3], [0, 3], [3, -1], [2, 0], [-1, -1]]
    assert np.allclose(wk, [[0.9, 0.8], [0.9, 0.8], [0.95, 0.0], [0.95, 0.8], [0.0, 0.0]])


def test_empty_and_single_edge():
    e = np.zeros(0, dtype=np.int32)
    rp, col, w = oracle.graph_csr(e, e, np.zeros(0, np.float32), 3)
    assert rp.tolist() == [0, 0, 0, 0] and col.size == 0
    rp, col, w = oracle.graph_csr(np.array([0]), np.array([1]), np.array([0.7], np.float32), 2)
    assert rp.tolist() == [0, 1, 2] and col.tolist() == [1, 0]


@pytest.mark.parametrize("n,count,skew", [(50, 200, 0.0), (2000, 20000, 1.1), (300, 40000, 0.5)])
def test_graph_matches_scipy_symmetrised_coo(n, count, skew):
    sp = pytest.importorskip("scipy.sparse")
    i, j, s = synth.pair_list(n, count, seed=n + count, skew=skew)
    rp, col, w = oracle.graph_csr(i, j, s, n)
    A = sp.coo_matrix((s, (i, j)), shape=(n, n))
    B = (A + A.T).tocsr()
    B.sort_indices()
    assert np.array_equal(rp, B.indptr)
    assert np.array_equal(col, B.indices)
    assert np.array_equal(w, B.data.astype(np.float32))
    # invariants: symmetric, degrees sum to twice the pairs
    assert rp[-1] == 2 * len(i)


def test_knn_matches_heap_selection():
    n = 400
    i, j, s = synth.pair_list(n, 6000, seed=7, skew=0.8)
    # quantise weights so that ties occur
    s = (np.round(s * 20) / 20).astype(np.float32)
    rp, col, w = oracle.graph_csr(i, j, s, n)
    for k in (1, 3, 17):
        nbr, wk = oracle.graph_knn(rp, col, w, k)
        for v in range(n):
            row = [(-float(w[q]), int(col[q])) for q in range(rp[v], rp[v + 1])]
            top = heapq.nsmallest(k, row)
            want_ids = [c for _, c in top] + [-1] * (k - len(top))
            want_w = [-x for x, _ in top] + [0.0] * (k - len(top))
            assert nbr[v].tolist() == want_ids
            assert np.allclose(wk[v], want_w)


def test_pair_list_generator_form():
    i, j, s = synth.pair_list(1000, 5000, seed=3, skew=1.0)
    key = i.astype(np.int64) * 1000 + j
    assert np.all(i < j) and np.all(np.diff(key) > 0) and np.all((s >= 0.5) & (s < 1.0))
    assert i.dtype == np.int32 and j.dtype == np.int32 and s.dtype == np.float32
