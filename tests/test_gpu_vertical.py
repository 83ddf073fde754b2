"""GPU parity of the vertical algorithm with local pruning (Sec. 5.1, Lemma 1, Eq. 2):
the exact candidate merge (aps_pairs_verify) against the oracle's float64 dots, and the
whole vertical join against the oracle's brute force for several block counts; plus the
sub-unit-norm join the blocks run on."""
import numpy as np
import pytest

import oracle
import synth
from parity import compare, row_dot64

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


def host_pairs(i, j):
    """A host aps_pairs view of two int32 arrays (kept alive by the caller)."""
    import ctypes

    import paper_1402_3010_gb300 as A

    p = A.aps_pairs()
    p.count = i.size
    p.i = i.ctypes.data_as(ctypes.c_void_p)
    p.j = j.ctypes.data_as(ctypes.c_void_p)
    p.score = None
    p.on_device = 0
    return p


def test_pairs_verify_against_oracle_dots(aps):
    c, _ = synth.config_small(seed=9, n=2000, m=3000)
    t = f32(0.3)
    # candidates: a seeded pair list with repeats across two lists
    i1, j1, _ = synth.pair_list(c.n, 60000, seed=1, skew=0.5)
    i2, j2, _ = synth.pair_list(c.n, 60000, seed=2, skew=0.5)
    ref = oracle.bruteforce(c, t)
    # add every true match to the second list so the result is the full match set
    i2 = np.concatenate([i2, ref.i.astype(np.int32)])
    j2 = np.concatenate([j2, ref.j.astype(np.int32)])
    lists = [host_pairs(i1, j1), host_pairs(i2, j2)]
    out, nc = aps.aps_pairs_verify(lists, c.indptr, c.idx, c.val, c.n, c.m, t)
    try:
        i, j, s = aps.pairs_to_numpy(out)
    finally:
        aps.aps_pairs_free(out)
    keys = np.unique(np.concatenate([i1.astype(np.int64) * c.n + j1, i2.astype(np.int64) * c.n + j2]))
    assert nc == keys.size
    compare(i, j, s, ref, t, c.n, csr=c)


def test_pairs_verify_rejects_bad_pairs(aps):
    import paper_1402_3010_gb300 as A

    c, _ = synth.config_small(seed=9, n=50, m=300)
    i = np.array([3, 7], np.int32)
    j = np.array([9, 7], np.int32)  # 7 >= 7: not i < j
    with pytest.raises(A.APSError) as e:
        aps.aps_pairs_verify([host_pairs(i, j)], c.indptr, c.idx, c.val, c.n, c.m, 0.5)
    assert e.value.status == A.EINVAL


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_vertical_join_matches_oracle(aps, p):
    from paper_1402_3010_gb300 import vertical as V

    rng = np.random.default_rng(21)
    lengths = synth.power_law_lengths(rng, 4000, synth.ALPHA_MEAN50, 1, 300)
    c = synth.sparse_vectors(4000, 2500, lengths, 1.0, "lognormal", 21, rng=rng)
    t = f32(0.6)
    out, info = V.vertical_all_pairs(c.indptr, c.idx, c.val, c.n, c.m, t, p)
    try:
        i, j, s = aps.pairs_to_numpy(out)
    finally:
        aps.aps_pairs_free(out)
    ref = oracle.bruteforce(c, t)
    r = compare(i, j, s, ref, t, c.n, csr=c)
    assert r["pairs"] > 0
    assert info["candidates"] >= len(i) and len(info["local_pairs"]) == p


def test_subunit_norm_join_matches_oracle_on_a_projection(aps):
    """A block's projection (norms below 1) joined at t/p with APS_SUBUNIT_NORMS."""
    import torch

    import paper_1402_3010_gb300 as A
    from paper_1402_3010_gb300 import vertical as V

    c, _ = synth.config_small(seed=10, n=3000, m=2500)
    block = V.partition_dims(np.bincount(c.idx, minlength=c.m), 2)
    ip, ix, vv = V.project(c.indptr, c.idx, c.val, block, 1)
    proj = synth.SparseCSR(ip, ix, vv, c.n, c.m)
    tl = V.local_threshold(0.6, 2)
    h = A.aps_build_index(*(torch.from_numpy(a).cuda() for a in (ip, ix, vv)), c.n, c.m, tl, A.SUBUNIT_NORMS)
    try:
        p = A.aps_all_pairs(h)
        i, j, s = A.pairs_to_numpy(p)
        A.aps_pairs_free(p)
    finally:
        A.aps_index_free(h)
    compare(i, j, s, oracle.bruteforce(proj, f32(tl)), f32(tl), c.n, csr=proj)
    # without the flag the projection is rejected (norms below 1)
    with pytest.raises(A.APSError) as e:
        A.aps_build_index(ip, ix, vv, c.n, c.m, tl)
    assert e.value.status == A.EINVAL


# ----------------------------------------------- the local pruning inside the join


@pytest.mark.parametrize("nblk,heavy,t", [(2, 300, 0.7), (4, 300, 0.6), (3, 10**9, 0.7), (2, 50, 0.9)])
def test_split_join_matches_oracle_and_plain_join(aps, nblk, heavy, t):
    """aps_all_pairs_split: the `heavy` costliest vectors joined as nblk dimension blocks with
    the local threshold of Lemma 1 inside the join, every pair decided exactly; the pair set
    is the oracle's (and the plain join's) and the output stays in (i, j) order."""
    import paper_1402_3010_gb300 as A

    rng = np.random.default_rng(90 + nblk)
    lengths = synth.power_law_lengths(rng, 24000, synth.ALPHA_MEAN50, 1, 600)
    c = synth.sparse_vectors(24000, 6000, lengths, 1.0, "lognormal", 90 + nblk, rng=rng)
    tt = f32(t)
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, tt)
    try:
        p = A.aps_all_pairs_split(h, nblk, heavy)
        try:
            i, j, s = A.pairs_to_numpy(p)
        finally:
            A.aps_pairs_free(p)
        st = A.aps_index_stats(h)
        q = A.aps_all_pairs(h)
        try:
            pi, pj, ps = A.pairs_to_numpy(q)
        finally:
            A.aps_pairs_free(q)
    finally:
        A.aps_index_free(h)
    r = compare(i, j, s, oracle.bruteforce(c, tt), tt, c.n, csr=c)
    assert r["pairs"] > 0 and st["pairs"] == len(i)
    # the split changes the work, not the pairs: identical to the plain join outside the band
    keys = i.astype(np.int64) * c.n + j
    pkeys = pi.astype(np.int64) * c.n + pj
    diff = np.setxor1d(keys, pkeys)
    for k in diff.tolist():
        assert abs(row_dot64(c, *divmod(k, c.n)) - tt) <= 1e-5


def test_split_join_rejects_bad_arguments(aps):
    import paper_1402_3010_gb300 as A

    c, t = synth.config_small(seed=1)
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    try:
        for nblk, heavy in ((1, 10), (9, 10), (2, -1)):
            with pytest.raises(A.APSError) as e:
                A.aps_all_pairs_split(h, nblk, heavy)
            assert e.value.status == A.EINVAL
        p = A.aps_all_pairs_split(h, 2, 0)  # no heavy vector: the plain join
        try:
            i, j, s = A.pairs_to_numpy(p)
        finally:
            A.aps_pairs_free(p)
        compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), c.n, csr=c)
    finally:
        A.aps_index_free(h)
