"""GPU checks of the join's tile shapes: every shape gives the oracle's pairs, and the
autotuner's table changes the join time only."""
import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch

    import paper_1402_3010_gb300 as A
    from paper_1402_3010_gb300 import _build

    _build.build()
    A.load()
    torch.cuda.init()
    yield A
    A.aps_set_tuning(A.aps_tuning_default())


def _instance(c, ro, m, r):
    a, b = int(ro[r]), int(ro[r + 1])
    ip = c.indptr[a:b + 1] - c.indptr[a]
    return synth.SparseCSR(ip, c.idx[c.indptr[a]:c.indptr[b]], c.val[c.indptr[a]:c.indptr[b]], b - a, int(m[r]))


def _run(A, ro, dev, m, ts):
    outs, st = A.aps_batch_all_pairs_csr(ro, *dev, m, ts)
    try:
        res = [A.pairs_to_numpy(o) for o in outs]
    finally:
        for o in outs:
            A.aps_pairs_free(o)
    return res, st


def test_every_tile_shape_matches_the_oracle(A):
    """One batch (n from 3 to 14000: one window at G = 8 up to 5120 vectors, up to three
    windows at G = 8 above) joined with G = 1, 2, 4 and 8 forced for every instance."""
    import torch

    rng = np.random.default_rng(81)
    k = 24
    ns = np.exp(rng.uniform(np.log(3), np.log(14000), size=k)).astype(np.int64)
    ns[[3, 11]] = [5120, 5121]  # both sides of the one-window bound at G = 8
    ts = rng.uniform(0.6, 0.9, size=k).astype(np.float32)
    lengths = synth.poisson_lengths(rng, int(ns.sum()), 10, 1, 60)
    c = synth.sparse_vectors(int(ns.sum()), 2000, lengths, 1.1, "uniform", 81, rng=rng)
    ro = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    m = np.full(k, 2000, np.int32)
    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    refs = [oracle.bruteforce(_instance(c, ro, m, r), float(ts[r])) for r in range(k)]
    try:
        for g in (1, 2, 4, 8):
            A.aps_set_tuning([g] * A.TUNE_BUCKETS)
            res, st = _run(A, ro, dev, m, ts)
            assert st["pairs"] == sum(len(x[0]) for x in res)
            for r in range(k):
                i, j, s = res[r]
                compare(i, j, s, refs[r], float(ts[r]), max(int(ns[r]), 1), csr=_instance(c, ro, m, r))
    finally:
        A.aps_set_tuning(A.aps_tuning_default())


def test_autotuner_measures_every_populated_bucket_and_keeps_results(A):
    """The batched workload's generator (64 instances, n log-uniform in [100, 20000]):
    the tuner times each populated bucket under the four shapes, installs a valid table,
    and the batch's pairs under that table equal those under the default table."""
    import torch

    ro, c, m, ts = synth.config_batched_csr(k=64)
    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    try:
        A.aps_set_tuning(A.aps_tuning_default())
        base, _ = _run(A, ro, dev, m, ts)
        groups, rep = A.aps_autotune_batch_csr(ro, *dev, m, ts)
        assert A.aps_get_tuning() == groups
        assert all(g in (1, 2, 4, 8) for g in groups)
        sizes = np.diff(ro)
        for b in range(A.TUNE_BUCKETS):
            want = int(sum(A.aps_tune_bucket(int(n)) == b for n in sizes))
            assert rep["instances"][b] == want
            if want:
                assert 1 <= rep["sampled"][b] <= want
                assert all(v > 0 for v in rep["ms"][b])
            else:
                assert rep["sampled"][b] == 0 and all(v == -1 for v in rep["ms"][b])
        assert rep["ms_default"] > 0 and rep["ms_tuned"] > 0
        if rep["ms_tuned"] >= rep["ms_default"]:
            assert groups == A.aps_tuning_default()
        tuned, _ = _run(A, ro, dev, m, ts)
        for r in range(len(sizes)):
            n = max(int(sizes[r]), 1)
            ka = base[r][0].astype(np.int64) * n + base[r][1]
            kb = tuned[r][0].astype(np.int64) * n + tuned[r][1]
            sa = dict(zip(ka.tolist(), base[r][2].tolist()))
            sb = dict(zip(kb.tolist(), tuned[r][2].tolist()))
            t = float(ts[r])
            assert all(abs(sa[q] - t) <= 1e-5 for q in set(sa) - set(sb))
            assert all(abs(sb[q] - t) <= 1e-5 for q in set(sb) - set(sa))
            assert all(abs(sa[q] - sb[q]) <= 1e-5 for q in set(sa) & set(sb))
    finally:
        A.aps_set_tuning(A.aps_tuning_default())


def test_repeated_joins_of_one_index_replay_the_join_graph(A):
    """The first join of an index captures its join phase as a CUDA graph; later joins
    replay it with their own buffers (new staging and count arrays each time), with the
    same pairs as the first join and as the oracle. Join flags may change between joins."""
    import torch

    rng = np.random.default_rng(83)
    lengths = synth.power_law_lengths(rng, 3000, synth.ALPHA_MEAN50, 1, 300)
    c = synth.sparse_vectors(3000, 2500, lengths, 1.0, "lognormal", 83, rng=rng)
    t = float(np.float32(0.6))
    ip, ix, vv = (torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val))
    ref = oracle.bruteforce(c, t)
    h = A.aps_build_index(ip, ix, vv, c.n, c.m, t, 0)
    try:
        runs = []
        for flags in (0, 0, A.NO_UPPERBOUND, 0):
            p = A.aps_all_pairs(h, flags)
            try:
                runs.append(A.pairs_to_numpy(p))
            finally:
                A.aps_pairs_free(p)
        for i, j, s in runs:
            compare(i, j, s, ref, t, c.n, csr=c)
            assert np.array_equal(i, runs[0][0]) and np.array_equal(j, runs[0][1])
        assert len(runs[0][0]) > 100
    finally:
        A.aps_index_free(h)


def test_staging_overflow_grows_and_reruns_the_join(A):
    """A join whose staging room is far too small (test hook: room for 1000 pairs) sees
    its slab reservations exceed the room, grows the buffer and runs again: one re-run,
    the oracle's pairs. The re-run replays the join graph with the new buffer."""
    import torch

    rng = np.random.default_rng(85)
    lengths = synth.power_law_lengths(rng, 4000, synth.ALPHA_MEAN50, 1, 300)
    c = synth.sparse_vectors(4000, 3000, lengths, 1.0, "lognormal", 85, rng=rng)
    t = float(np.float32(0.6))
    ip, ix, vv = (torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val))
    ref = oracle.bruteforce(c, t)
    assert len(ref.i) > 20_000
    h = A.aps_build_index(ip, ix, vv, c.n, c.m, t, 0)
    try:
        for cap in (1000, 0):  # an overflowing join, then one with the estimate from it
            A.aps_debug_stage_cap(cap)
            p = A.aps_all_pairs(h)
            try:
                i, j, s = A.pairs_to_numpy(p)
            finally:
                A.aps_pairs_free(p)
            st = A.aps_index_stats(h)
            assert st["reruns"] == (1 if cap else 0)
            compare(i, j, s, ref, t, c.n, csr=c)
    finally:
        A.aps_debug_stage_cap(0)
        A.aps_index_free(h)


def test_every_query_tile_shape_matches_the_oracle(A):
    """A queryable index of 30000 vectors (three windows at G = 2, one at G = 1, six at
    G = 8) built under each G of the queryable column, queried with 300 rows of the same
    power-law family: the oracle's cross pairs every time."""
    m = 12000
    perm = np.random.default_rng(2087).permutation(m)
    r1 = np.random.default_rng(87)
    c = synth.sparse_vectors(30000, m, synth.power_law_lengths(r1, 30000, synth.ALPHA_MEAN40, 1, 300), 1.0,
                             "lognormal", 87, rng=r1, perm=perm)
    r2 = np.random.default_rng(88)
    q = synth.sparse_vectors(300, m, synth.power_law_lengths(r2, 300, synth.ALPHA_MEAN40, 1, 300), 1.0,
                             "lognormal", 88, rng=r2, perm=perm)
    t = float(np.float32(0.7))
    ref = oracle.bruteforce_cross(q, c, t)
    assert len(ref.i) > 100
    default_q = A.aps_tuning_default(query=True)
    try:
        for g in (1, 2, 4, 8):
            A.aps_set_tuning(A.aps_tuning_default(), [g] * A.TUNE_BUCKETS)
            h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t, A.QUERYABLE)
            try:
                p = A.aps_query(h, q.indptr, q.idx, q.val, q.n, t)
                try:
                    i, j, s = A.pairs_to_numpy(p)
                finally:
                    A.aps_pairs_free(p)
            finally:
                A.aps_index_free(h)
            compare(i, j, s, ref, t, c.n, self_join=False, csr=c, queries=q)
    finally:
        A.aps_set_tuning(A.aps_tuning_default(), default_q)
