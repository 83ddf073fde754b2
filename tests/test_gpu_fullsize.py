"""Parity at the stated sizes of the workloads (the problem definition of Sec. 2.1: every
pair with dot >= t, once, as i < j), against the CPU oracle run on every host core:

- the 200k x 100k power-law set at t = 0.7: the whole pair set (about 9.7e7 pairs) against
  the oracle's all-pairs-2 (Alg. 1-2 with the all-pairs-1/2 bounds);
- the 512-instance batched set, every instance;
- a second 512-instance batched set drawn from the large set's family, which has matches;
- query batches against the 1M-vector serving index (64 sampled queries), directly and
  through the serving loop.
Pairs only the GPU reports are judged by their float64 score recomputed from the inputs."""
import numpy as np
import pytest

import oracle
import synth
from oracle_pool import all_pairs_parallel, instances_parallel
from parity import compare, compare_large, row_dot64

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


def test_large_set_whole_pair_set(aps):
    import torch

    c = synth.config_large()
    t = f32(0.7)
    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    h = aps.aps_build_index(*dev, c.n, c.m, t)
    try:
        p = aps.aps_all_pairs(h)
        try:
            gi, gj, gs = aps.pairs_to_numpy(p)
        finally:
            aps.aps_pairs_free(p)
    finally:
        aps.aps_index_free(h)
    del dev
    ri, rj, rs = all_pairs_parallel(c, t)
    r = compare_large(gi, gj, gs, ri, rj, rs, t, c.n, lambda a, b: row_dot64(c, a, b))
    assert r["pairs"] > 90_000_000 and r["ref"] > 90_000_000


def _instance(c, ro, m, r):
    a, b = int(ro[r]), int(ro[r + 1])
    return synth.SparseCSR(c.indptr[a:b + 1] - c.indptr[a], c.idx[c.indptr[a]:c.indptr[b]],
                           c.val[c.indptr[a]:c.indptr[b]], b - a, int(m[r]))


def _batch_against_oracle(aps, ro, c, m, ts):
    import torch

    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    outs, st = aps.aps_batch_all_pairs_csr(ro, *dev, m, ts)
    try:
        got = [aps.pairs_to_numpy(o) for o in outs]
    finally:
        for o in outs:
            aps.aps_pairs_free(o)
    refs = instances_parallel(ro, c, m, ts)
    assert len(refs) == len(got) == len(ro) - 1
    total = 0
    for r, ((gi, gj, gs), (ri, rj, rs)) in enumerate(zip(got, refs)):
        cr = _instance(c, ro, m, r)
        compare_large(gi, gj, gs, ri, rj, rs, float(ts[r]), max(cr.n, 1), lambda a, b: row_dot64(cr, a, b))
        total += len(gi)
    assert total == st["pairs"]
    return total, sum(len(x[0]) for x in refs)


def test_batched_set_every_instance(aps):
    """All 512 instances of the batched set (n log-uniform in [100, 20000], Poisson(30)
    lengths, t ~ U(0.6, 0.9)). Its vectors rarely reach t: the whole batch has a handful of
    pairs, and every instance is compared, including the empty ones."""
    ro, c, m, ts = synth.config_batched_csr()
    got, ref = _batch_against_oracle(aps, ro, c, m, ts)
    assert got == ref


def test_batched_set_with_matches_every_instance(aps):
    """The second batched set (same sizes and thresholds, vectors from the large set's
    power-law family): millions of pairs, every instance compared."""
    ro, c, m, ts = synth.config_batched_matches()
    got, ref = _batch_against_oracle(aps, ro, c, m, ts)
    assert got > 1_000_000 and abs(got - ref) <= max(10, ref // 100000)


def test_serving_index_of_1m_vectors_sampled_queries(aps):
    import time

    import torch

    import paper_1402_3010_gb300 as A

    c, t = synth.config_serving()
    t = f32(t)
    q = synth.serving_queries(64)
    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    h = A.aps_build_index(*dev, c.n, c.m, t, A.QUERYABLE)
    try:
        p = A.aps_query(h, q.indptr, q.idx, q.val, q.n, t)
        try:
            i, j, s = A.pairs_to_numpy(p)
        finally:
            A.aps_pairs_free(p)
        # the same queries through the serving loop, four batches of 16 on two slots
        sv = A.aps_server_create(h, 8 << 30, 2)
        try:
            tickets = []
            for a in range(0, 64, 16):
                sub = synth.SparseCSR(q.indptr[a:a + 17] - q.indptr[a], q.idx[q.indptr[a]:q.indptr[a + 16]],
                                      q.val[q.indptr[a]:q.indptr[a + 16]], 16, q.m)
                tickets.append((a, A.aps_stream_submit(sv, sub.indptr, sub.idx, sub.val, 16, t)))
            parts = []
            deadline = time.time() + 300
            for a, tk in tickets:
                r = None
                while r is None and time.time() < deadline:
                    r = A.aps_stream_poll(sv, tk, 100000)
                assert r is not None
                x = A.pairs_to_numpy(r)
                A.aps_pairs_free(r)
                parts.append((x[0] + a, x[1], x[2]))
        finally:
            A.aps_server_free(sv)
    finally:
        A.aps_index_free(h)
    ref = oracle.bruteforce_cross(q, c, t)
    r = compare(i, j, s, ref, t, c.n, self_join=False, csr=c, queries=q)
    assert r["pairs"] > 0
    si = np.concatenate([x[0] for x in parts])
    sj = np.concatenate([x[1] for x in parts])
    ss = np.concatenate([x[2] for x in parts])
    assert np.array_equal(si, i) and np.array_equal(sj, j) and np.abs(ss - s).max(initial=0.0) <= 1e-5
