"""Fault injection into the serving loop (continuous batching of query batches against a
resident index, the local matching of Alg. 6), all on the host side: a device allocation
that fails inside one batch (the library's allocation hook), a malformed batch, batches
that are canceled or abandoned by their client, and a client thread that dies mid-stream.
Each fault must stay inside its own batch: every other batch returns exactly what the same
queries return alone, and the server keeps serving."""
import threading
import time

import numpy as np
import pytest

from test_gpu_serving import family, query, sub

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch

    import paper_1402_3010_gb300 as aps
    from paper_1402_3010_gb300 import _build

    _build.build()
    aps.load()
    torch.cuda.init()
    return aps


@pytest.fixture(scope="module")
def setup(A):
    c, q = family(8000, 400, 4000, seed=17)
    t = 0.7
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t, A.QUERYABLE)
    batches = [sub(q, a, a + 100) for a in range(0, 400, 100)]
    refs = [query(A, h, b, t) for b in batches]
    assert sum(len(r[0]) for r in refs) > 0
    yield h, t, batches, refs
    A.aps_index_free(h)


def wait(A, sv, tk, limit_s=60):
    deadline = time.time() + limit_s
    while time.time() < deadline:
        p = A.aps_stream_poll(sv, tk, 10000)
        if p is not None:
            try:
                return A.pairs_to_numpy(p)
            finally:
                A.aps_pairs_free(p)
    raise AssertionError("batch not done in time")


def same(got, ref):
    return np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]) and np.allclose(got[2], ref[2])


def submit(A, sv, b, t):
    return A.aps_stream_submit(sv, b.indptr, b.idx, b.val, b.n, t)


def test_allocation_failure_fails_only_its_batch(A, setup):
    h, t, batches, refs = setup
    sv = A.aps_server_create(h, 0, 1)  # one slot: the batches run one after another
    try:
        assert same(wait(A, sv, submit(A, sv, batches[0], t)), refs[0])
        A.aps_debug_fail_alloc(1)  # the next device allocation (inside the next batch) fails
        tk = submit(A, sv, batches[1], t)
        with pytest.raises(A.APSError) as e:
            wait(A, sv, tk)
        assert e.value.status == A.ENOMEM
        for k in (2, 3, 1):  # the server goes on, the failed batch included when resent
            assert same(wait(A, sv, submit(A, sv, batches[k], t)), refs[k])
    finally:
        A.aps_debug_fail_alloc(0)
        A.aps_server_free(sv)


def test_malformed_batch_fails_alone(A, setup):
    h, t, batches, refs = setup
    sv = A.aps_server_create(h, 8 << 30, 2)
    try:
        bad = batches[2]
        idx = bad.idx.copy()
        idx[len(idx) // 2] = 10 ** 6  # a dimension outside [0, m)
        tks = [submit(A, sv, batches[0], t)]
        try:
            tb = A.aps_stream_submit(sv, bad.indptr, idx, bad.val, bad.n, t)
        except A.APSError as err:  # rejected at submission
            assert err.status == A.EINVAL
            tb = None
        tks.append(submit(A, sv, batches[3], t))
        if tb is not None:
            with pytest.raises(A.APSError) as e:
                wait(A, sv, tb)
            assert e.value.status == A.EINVAL
        assert same(wait(A, sv, tks[0]), refs[0]) and same(wait(A, sv, tks[1]), refs[3])
    finally:
        A.aps_server_free(sv)


def test_canceled_and_abandoned_batches_release_the_server(A, setup):
    h, t, batches, refs = setup
    sv = A.aps_server_create(h, 1, 2)  # a 1-byte budget: one batch admitted at a time
    tks = [submit(A, sv, batches[k % 4], t) for k in range(8)]
    for tk in tks[4:6]:
        A.aps_stream_cancel(sv, tk)
    assert same(wait(A, sv, tks[0]), refs[0])
    t0 = time.time()
    A.aps_server_free(sv)  # the other batches are abandoned: running ones finish, queued ones drop
    assert time.time() - t0 < 60
    sv = A.aps_server_create(h, 8 << 30, 2)
    try:
        got = [wait(A, sv, tk) for tk in [submit(A, sv, b, t) for b in batches]]
        assert all(same(g, r) for g, r in zip(got, refs))
    finally:
        A.aps_server_free(sv)


def test_a_client_dying_mid_stream_leaves_the_others_served(A, setup):
    h, t, batches, refs = setup
    sv = A.aps_server_create(h, 8 << 30, 4)
    results, errors = {}, []

    def client(k, die):
        try:
            mine = [(j, submit(A, sv, batches[j], t)) for j in range(4)]
            if die:
                raise RuntimeError("client died")  # its tickets are never polled
            results[k] = [(j, wait(A, sv, tk)) for j, tk in mine]
        except RuntimeError as e:
            errors.append((k, str(e)))

    try:
        th = [threading.Thread(target=client, args=(k, k == 1)) for k in range(3)]
        for x in th:
            x.start()
        for x in th:
            x.join(120)
        assert errors == [(1, "client died")]
        assert sorted(results) == [0, 2]
        for k in (0, 2):
            for j, got in results[k]:
                assert same(got, refs[j])
    finally:
        A.aps_server_free(sv)
