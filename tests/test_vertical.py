"""Host logic of the vertical algorithm (Sec. 5.1): the first-fit dimension partition,
the projections, the local threshold, and Lemma 1 itself checked with the oracle (every
match reaches t/p on at least one block's projection)."""
import numpy as np
import pytest

import oracle
import synth


def test_partition_is_first_fit_by_quadratic_load():
    from paper_1402_3010_gb300 import vertical as V

    nnz = np.array([5, 1, 9, 3, 9, 0, 2])
    block = V.partition_dims(nnz, 2)
    # densest first (9 @2, 9 @4 by id), each into the least loaded block
    w = nnz * (nnz + 1) // 2
    load = [0, 0]
    want = np.empty(7, np.int32)
    for d in [2, 4, 0, 3, 6, 1, 5]:
        k = int(np.argmin(load))
        want[d] = k
        load[k] += w[d]
    assert np.array_equal(block, want)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_projections_partition_every_row(p):
    from paper_1402_3010_gb300 import vertical as V

    c, _ = synth.config_small(seed=7, n=300, m=800)
    block = V.partition_dims(np.bincount(c.idx, minlength=c.m), p)
    parts = [V.project(c.indptr, c.idx, c.val, block, k) for k in range(p)]
    for x in range(c.n):
        ids = np.sort(np.concatenate([ix[ip[x]:ip[x + 1]] for ip, ix, _ in parts]))
        assert np.array_equal(ids, c.idx[c.indptr[x]:c.indptr[x + 1]])
        ss = sum(float(np.sum(vv[ip[x]:ip[x + 1]].astype(np.float64) ** 2)) for ip, _, vv in parts)
        assert abs(ss - float(np.sum(c.val[c.indptr[x]:c.indptr[x + 1]].astype(np.float64) ** 2))) < 1e-9


def test_local_threshold_is_at_most_t_over_p():
    from paper_1402_3010_gb300 import vertical as V

    for t in (0.5, 0.7, 0.9, 0.123456):
        for p in (1, 2, 3, 4, 7):
            tl = V.local_threshold(t, p)
            assert tl <= t / p and tl > t / p * (1 - 1e-5)
            assert float(np.float32(tl)) == tl


@pytest.mark.parametrize("p", [2, 3, 4])
def test_lemma1_union_of_local_matches_holds_every_match(p):
    """Lemma 1 (Sec. 5.1): M(D, t) is contained in the union over blocks of M(D_k, t/p)."""
    from paper_1402_3010_gb300 import vertical as V

    c, _ = synth.config_small(seed=8, n=1500, m=2000)
    t = 0.6
    full = oracle.bruteforce(c, t)
    block = V.partition_dims(np.bincount(c.idx, minlength=c.m), p)
    union = set()
    for k in range(p):
        ip, ix, vv = V.project(c.indptr, c.idx, c.val, block, k)
        r = oracle.bruteforce(synth.SparseCSR(ip, ix, vv, c.n, c.m), V.local_threshold(t, p))
        union.update((r.i.astype(np.int64) * c.n + r.j).tolist())
    keys = (full.i.astype(np.int64) * c.n + full.j).tolist()
    assert len(keys) > 0
    assert set(keys) <= union
    # and the pruning is real: the union is smaller than all pairs sharing a dimension
    assert len(union) < c.n * (c.n - 1) // 2
