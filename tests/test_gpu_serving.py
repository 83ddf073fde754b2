"""GPU parity of external queries (aps_query) and of the serving loop (continuous
batching): every result against the oracle's query-vs-set brute force, and each batch's
result alone equal to its result in a mix of concurrently running batches."""
import time

import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aps():
    import torch

    import paper_1402_3010_gb300 as aps
    from paper_1402_3010_gb300 import _build

    _build.build()
    aps.load()
    torch.cuda.init()
    return aps


def f32(t):
    return float(np.float32(t))


def family(n, nq, m, seed, hi=300):
    """An index set and a query set drawn from the same power-law family and sharing
    their dense dimensions (one rank -> id permutation)."""
    perm = np.random.default_rng(seed + 1000).permutation(m)
    r1 = np.random.default_rng(seed)
    c = synth.sparse_vectors(n, m, synth.power_law_lengths(r1, n, synth.ALPHA_MEAN40, 1, hi), 1.0, "lognormal",
                             seed, rng=r1, perm=perm)
    r2 = np.random.default_rng(seed + 1)
    q = synth.sparse_vectors(nq, m, synth.power_law_lengths(r2, nq, synth.ALPHA_MEAN40, 1, hi), 1.0, "lognormal",
                             seed + 1, rng=r2, perm=perm)
    return c, q


def query(aps, h, q, t, flags=0):
    p = aps.aps_query(h, q.indptr, q.idx, q.val, q.n, t, flags)
    try:
        return aps.pairs_to_numpy(p)
    finally:
        aps.aps_pairs_free(p)


def sub(q, a, b):
    ip = q.indptr[a:b + 1] - q.indptr[a]
    return synth.SparseCSR(ip.astype(np.int64), q.idx[q.indptr[a]:q.indptr[b]], q.val[q.indptr[a]:q.indptr[b]],
                           b - a, q.m)


@pytest.mark.parametrize("n,t_build,t_query", [(6000, 0.6, 0.6), (6000, 0.5, 0.75), (45000, 0.7, 0.7)])
def test_query_parity(aps, n, t_build, t_query):
    import paper_1402_3010_gb300 as A

    c, q = family(n, 400, 3000 if n < 10000 else 15000, seed=n)
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t_build, A.QUERYABLE)
    try:
        i, j, s = query(aps, h, q, t_query)
    finally:
        A.aps_index_free(h)
    ref = oracle.bruteforce_cross(q, c, f32(t_query))
    r = compare(i, j, s, ref, f32(t_query), c.n, self_join=False, csr=c, queries=q)
    assert r["pairs"] > 0


def test_query_rejects_unqueryable_index_and_low_threshold(aps):
    import paper_1402_3010_gb300 as A

    c, q = family(2000, 10, 1500, seed=3)
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, 0.7)
    try:
        with pytest.raises(A.APSError) as e:
            query(aps, h, q, 0.7)
        assert e.value.status == A.EINVAL and "QUERYABLE" in str(e.value)
    finally:
        A.aps_index_free(h)
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, 0.7, A.QUERYABLE)
    try:
        with pytest.raises(A.APSError) as e:
            query(aps, h, q, 0.6)
        assert e.value.status == A.EINVAL
    finally:
        A.aps_index_free(h)


def test_self_join_on_queryable_index(aps):
    """The norm-bound prefix split is also valid for the self-join."""
    import paper_1402_3010_gb300 as A

    c, _ = family(5000, 1, 3000, seed=4)
    t = 0.6
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t, A.QUERYABLE)
    try:
        p = A.aps_all_pairs(h)
        i, j, s = A.pairs_to_numpy(p)
        A.aps_pairs_free(p)
    finally:
        A.aps_index_free(h)
    compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), c.n, csr=c)


def test_serving_results_alone_equal_results_in_the_mix(aps):
    import paper_1402_3010_gb300 as A

    c, q = family(30000, 1200, 8000, seed=5)
    t = 0.75
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t, A.QUERYABLE)
    try:
        rng = np.random.default_rng(6)
        bounds, a = [], 0
        while a < q.n:
            b = min(q.n, a + int(np.exp(rng.uniform(0, np.log(300)))))
            bounds.append((a, b))
            a = b
        alone = [query(aps, h, sub(q, a, b), t) for a, b in bounds]
        sv = A.aps_server_create(h, 8 << 30, 4)
        try:
            tickets = []
            for a, b in bounds:  # all submitted at once: batches run concurrently on 4 slots
                qb = sub(q, a, b)
                tickets.append(A.aps_stream_submit(sv, qb.indptr, qb.idx, qb.val, qb.n, t))
            mixed = [None] * len(tickets)
            deadline = time.time() + 120
            while any(m is None for m in mixed) and time.time() < deadline:
                for k, tk in enumerate(tickets):
                    if mixed[k] is None:
                        p = A.aps_stream_poll(sv, tk, 1000)
                        if p is not None:
                            assert p.on_device == 0
                            mixed[k] = A.pairs_to_numpy(p)
                            A.aps_pairs_free(p)
            assert all(m is not None for m in mixed)
            # the batches ran side by side on the device, not one after another
            st = A.aps_server_timeline(sv)
            assert st["batches"] == len(bounds)
            assert st["max_in_flight"] >= 2 and st["overlap_ms"] > 0.0
            assert 0.0 < st["busy_ms"] <= st["span_ms"] + 1e-3
        finally:
            A.aps_server_free(sv)
    finally:
        A.aps_index_free(h)
    for (a, b), x, y in zip(bounds, alone, mixed):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert np.abs(x[2] - y[2]).max(initial=0.0) <= 1e-5
    # and the union is the oracle's answer
    I = np.concatenate([x[0] + a for (a, _), x in zip(bounds, mixed)])
    J = np.concatenate([x[1] for x in mixed])
    S = np.concatenate([x[2] for x in mixed])
    compare(I, J, S, oracle.bruteforce_cross(q, c, f32(t)), f32(t), c.n, self_join=False, csr=c, queries=q)


def test_serving_cancel_budget_and_errors(aps):
    import paper_1402_3010_gb300 as A

    c, q = family(8000, 300, 4000, seed=7)
    t = 0.7
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t, A.QUERYABLE)
    try:
        ref = query(aps, h, q, t)
        sv = A.aps_server_create(h, 1, 1)  # budget of 1 byte: one batch at a time
        try:
            tk = [A.aps_stream_submit(sv, q.indptr, q.idx, q.val, q.n, t) for _ in range(3)]
            A.aps_stream_cancel(sv, tk[2])
            for k in range(2):
                p = None
                deadline = time.time() + 60
                while p is None and time.time() < deadline:
                    p = A.aps_stream_poll(sv, tk[k], 10000)
                got = A.pairs_to_numpy(p)
                A.aps_pairs_free(p)
                assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
            with pytest.raises(A.APSError) as e:
                deadline = time.time() + 60
                while time.time() < deadline:
                    if A.aps_stream_poll(sv, tk[2], 10000) is not None:
                        break
            assert e.value.status == A.ECANCELED
            with pytest.raises(A.APSError) as e:
                A.aps_stream_poll(sv, 999999, 0)
            assert e.value.status == A.EINVAL
            with pytest.raises(A.APSError) as e:
                A.aps_stream_submit(sv, q.indptr, q.idx, q.val, q.n, 0.5)
            assert e.value.status == A.EINVAL
        finally:
            A.aps_server_free(sv)
    finally:
        A.aps_index_free(h)


def test_serving_shape_index_sampled_queries(aps):
    """The serving workload's generator (power law, mean 40, shared dense dimensions) with
    a 200k-vector queryable index at t = 0.75: 64 queries from the query generator against
    the oracle's float64 query-vs-set brute force."""
    import torch

    import paper_1402_3010_gb300 as A

    c, t = synth.config_serving(n=200_000)
    q = synth.serving_queries(64)
    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    h = A.aps_build_index(*dev, c.n, c.m, t, A.QUERYABLE)
    try:
        i, j, s = query(aps, h, q, t)
    finally:
        A.aps_index_free(h)
    ref = oracle.bruteforce_cross(q, c, f32(t))
    r = compare(i, j, s, ref, f32(t), c.n, self_join=False, csr=c, queries=q)
    assert r["pairs"] > 0
