"""GPU parity of the sparse path: every step of the index build and the self-join,
through the C ABI, against the CPU oracle on the same seeded inputs."""
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


def run_join(aps, c, t, build_flags=0, join_flags=0, device_input=True):
    import torch

    if device_input:
        ip, ix, vv = (torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val))
    else:
        ip, ix, vv = c.indptr, c.idx, c.val
    h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t, build_flags)
    try:
        p = aps.aps_all_pairs(h, join_flags)
        try:
            i, j, s = aps.pairs_to_numpy(p)
        finally:
            aps.aps_pairs_free(p)
        st = aps.aps_index_stats(h)
    finally:
        aps.aps_index_free(h)
    return i, j, s, st


def pl_small(seed, n, m, zipf=1.0, mean_alpha=synth.ALPHA_MEAN50, hi=300, weights="lognormal"):
    rng = np.random.default_rng(seed)
    lengths = synth.power_law_lengths(rng, n, mean_alpha, 1, min(hi, m))
    return synth.sparse_vectors(n, m, lengths, zipf, weights, seed, rng=rng)


# ------------------------------------------------------------------- self-join


def test_small_config_full_parity(aps):
    c, t = synth.config_small()
    i, j, s, st = run_join(aps, c, t)
    ref = oracle.bruteforce(c, f32(t))
    r = compare(i, j, s, ref, f32(t), c.n, csr=c)
    assert r["pairs"] > 0
    assert st["pairs"] == len(i)
    assert st["evaluations"] == c.n * (c.n - 1) // 2
    assert st["visits"] > 0 and st["candidates"] >= st["pairs"]


@pytest.mark.parametrize("seed,t", [(11, 0.5), (12, 0.7), (13, 0.9), (14, 0.3)])
def test_power_law_shapes_parity(aps, seed, t):
    c = pl_small(seed, n=3000, m=2000)
    i, j, s, _ = run_join(aps, c, t)
    compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), c.n, csr=c)


@pytest.mark.parametrize("n", [5121, 10241, 20481])
def test_every_group_class_and_ragged_sizes(aps, n):
    """Instance sizes just past each group-class boundary (8, 4, 2 and 1 query groups
    per CTA) with a ragged last window."""
    c = pl_small(20 + n % 7, n=n, m=4000, hi=60)
    t = 0.8
    i, j, s, _ = run_join(aps, c, t)
    ref, _ = oracle.all_pairs(c, f32(t), oracle.ALL_PAIRS_2)
    compare(i, j, s, ref, f32(t), c.n, csr=c)


def test_multi_window_instance(aps):
    """n > 40960: two candidate windows per early query, ragged second window."""
    c = pl_small(31, n=45000, m=20000, hi=40)
    t = 0.85
    i, j, s, st = run_join(aps, c, t)
    ref, _ = oracle.all_pairs(c, f32(t), oracle.ALL_PAIRS_2)
    compare(i, j, s, ref, f32(t), c.n, csr=c)


@pytest.mark.parametrize("t", [0.5, 0.8, 0.95])
@pytest.mark.parametrize("join_flags", [0, 0x10, 0x20, 0x70])
def test_one_and_two_component_vectors(aps, t, join_flags):
    """Vectors of one and two components (the streamed class: no accumulator, the two lists
    of a two-component vector merged by id) over several candidate windows (n > 20480), with
    dense dimensions so that lists are long, an id shared by both lists is common and
    two-component vectors often meet a rank in the other vector's unindexed prefix; the
    pruning toggles (remscore, minsize, upperbound off) change which vectors create."""
    rng = np.random.default_rng(91)
    n, m = 30000, 300
    lengths = rng.integers(1, 3, size=n)
    c = synth.sparse_vectors(n, m, lengths, 1.0, "lognormal", 91, rng=rng)
    i, j, s, st = run_join(aps, c, f32(t), 0, join_flags)
    ref, _ = oracle.all_pairs(c, f32(t), oracle.ALL_PAIRS_2)
    assert len(ref.i) > 1000
    compare(i, j, s, ref, f32(t), c.n, csr=c)
    assert st["visits"] <= st["entries_read"]


def test_short_vectors_among_long_ones_on_a_batch(aps):
    """A batch whose instances mix one- and two-component vectors with long ones: the
    streamed class and the windowed classes share one launch, each instance's pairs in its
    own output range."""
    import torch

    rng = np.random.default_rng(92)
    sizes = [700, 3000, 25000, 90]
    parts = []
    for k, n in enumerate(sizes):
        lengths = np.where(rng.random(n) < 0.5, rng.integers(1, 3, size=n), rng.integers(3, 60, size=n))
        parts.append(synth.sparse_vectors(n, 500, lengths, 1.0, "lognormal", 93 + k, rng=rng))
    ro = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ip = np.concatenate([[0]] + [p.indptr[1:] + sum(q.nnz for q in parts[:k]) for k, p in enumerate(parts)])
    ix = np.concatenate([p.idx for p in parts])
    vv = np.concatenate([p.val for p in parts])
    ts = np.array([0.6, 0.75, 0.9, 0.5], dtype=np.float32)
    outs, _ = aps.aps_batch_all_pairs_csr(ro, torch.from_numpy(ip.astype(np.int64)).cuda(),
                                          torch.from_numpy(ix).cuda(), torch.from_numpy(vv).cuda(),
                                          np.full(len(sizes), 500, np.int32), ts, 0)
    try:
        for k, (p, o) in enumerate(zip(parts, outs)):
            i, j, s = aps.pairs_to_numpy(o)
            ref, _ = oracle.all_pairs(p, float(ts[k]), oracle.ALL_PAIRS_2)
            compare(i, j, s, ref, float(ts[k]), p.n, csr=p)
    finally:
        for o in outs:
            aps.aps_pairs_free(o)


@pytest.mark.parametrize(
    "build_flags,join_flags",
    [(0, 0), (8, 0), (0, 0x10), (0, 0x20), (0, 0x40), (0, 0x70), (8, 0x70), (4, 0), (2, 0)],
)
def test_pruning_toggles_change_work_not_results(aps, build_flags, join_flags):
    import paper_1402_3010_gb300 as A

    c = pl_small(41, n=2500, m=1500)
    t = 0.6
    if build_flags & A.NORMALIZE:
        # scale rows away from unit norm; NORMALIZE must restore the same set
        c2 = synth.SparseCSR(c.indptr, c.idx, (c.val * 3.0).astype(np.float32), c.n, c.m)
        i, j, s, _ = run_join(aps, c2, t, build_flags, join_flags)
    else:
        i, j, s, _ = run_join(aps, c, t, build_flags, join_flags)
    compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), c.n, csr=c, tol=2e-5 if build_flags & 2 else 1e-5)


PAPER_VARIANTS = ["all-pairs-0-array", "all-pairs-0-remscore", "all-pairs-0-minsize", "all-pairs-1-array",
                  "all-pairs-1-remscore", "all-pairs-1-upperbound", "all-pairs-1-minsize",
                  "all-pairs-1-remscore-minsize", "all-pairs-2"]


@pytest.mark.parametrize("name", PAPER_VARIANTS)
def test_paper_variant_matches_oracle(aps, name):
    """Each of the paper's sequential variants (Sec. 4, Tables 2-3) returns the exact set."""
    import paper_1402_3010_gb300 as A

    c = pl_small(43, n=3000, m=1800)
    t = 0.6
    i, j, s, _ = run_join(aps, c, t, A.VARIANTS[name])
    compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), c.n, csr=c)


def test_paper_variants_only_remove_work(aps):
    """Every bound only removes work: partial indexing never adds posting visits, remscore
    never adds candidates, upperbound never adds prefix dots, minsize never adds candidates,
    a full index has no prefix dots, and every variant returns the same pairs."""
    import paper_1402_3010_gb300 as A

    c = pl_small(44, n=6000, m=3000)
    t = 0.7
    W, out = {}, {}
    for name in PAPER_VARIANTS:
        i, j, s, st = run_join(aps, c, t, A.VARIANTS[name])
        W[name] = st
        out[name] = (i.astype(np.int64) * c.n + j, s)
    assert W["all-pairs-1-array"]["visits"] <= W["all-pairs-0-array"]["visits"]
    assert W["all-pairs-0-remscore"]["candidates"] <= W["all-pairs-0-array"]["candidates"]
    assert W["all-pairs-1-remscore"]["candidates"] <= W["all-pairs-1-array"]["candidates"]
    assert W["all-pairs-0-minsize"]["candidates"] <= W["all-pairs-0-array"]["candidates"]
    assert W["all-pairs-1-minsize"]["candidates"] <= W["all-pairs-1-array"]["candidates"]
    assert W["all-pairs-1-upperbound"]["verified"] <= W["all-pairs-1-array"]["verified"]
    assert W["all-pairs-2"]["verified"] <= W["all-pairs-1-remscore-minsize"]["verified"]
    for name in PAPER_VARIANTS[:3]:
        assert W[name]["verified"] == 0
    # the bounds prune for real on this input
    assert W["all-pairs-2"]["candidates"] < W["all-pairs-1-array"]["candidates"]
    assert W["all-pairs-1-array"]["visits"] < W["all-pairs-0-array"]["visits"]
    k2, s2 = out["all-pairs-2"]
    assert len(k2) > 0
    for name in PAPER_VARIANTS:
        assert np.array_equal(out[name][0], k2), name
        assert np.abs(out[name][1] - s2).max(initial=0.0) <= 1e-5, name


def test_host_and_device_inputs_agree(aps):
    c, t = synth.config_small(seed=5, n=800, m=2000)
    a = run_join(aps, c, t, device_input=True)
    b = run_join(aps, c, t, device_input=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.allclose(a[2], b[2], atol=1e-6)


def test_host_output_flag(aps):
    import paper_1402_3010_gb300 as A

    c, t = synth.config_small(seed=6, n=700, m=1500)
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    try:
        p = A.aps_all_pairs(h, A.HOST_OUTPUT)
        assert p.on_device == 0
        i, j, s = A.pairs_to_numpy(p)
        A.aps_pairs_free(p)
    finally:
        A.aps_index_free(h)
    compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), c.n, csr=c)


def test_pair_set_is_deterministic(aps):
    c = pl_small(51, n=4000, m=2500)
    a = run_join(aps, c, 0.7)
    b = run_join(aps, c, 0.7)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.abs(a[2] - b[2]).max() <= 2e-6


# ------------------------------------------------------------------- edge cases


def csr_raw(rows, m):
    indptr = [0]
    idx, val = [], []
    for r in rows:
        for k in sorted(r):
            idx.append(k)
            val.append(r[k])
        indptr.append(len(idx))
    return synth.SparseCSR(np.array(indptr, np.int64), np.array(idx, np.int32), np.array(val, np.float32),
                           len(rows), m)


@pytest.mark.parametrize(
    "rows,m,t",
    [
        ([], 4, 0.5),  # empty set
        ([{1: 1.0}], 4, 0.5),  # one vector
        ([{}, {}, {}], 4, 0.5),  # only empty rows
        ([{2: 1.0}] * 50 + [{3: 1.0}] * 3, 5, 1.0),  # duplicates, t = 1
        ([{0: 1.0}, {0: 0.5, 1: 0.75}, {0: 0.5, 1: 0.25, 2: 0.75}, {1: 1.0}], 4, 0.5),  # exact ties
        ([{0: 0.6, 1: 0.8}, {}, {0: 0.8, 1: 0.6}, {}, {1: 1.0}], 3, 0.96),
    ],
)
def test_degenerate_inputs(aps, rows, m, t):
    c = csr_raw(rows, m)
    if c.nnz:
        nrm = np.sqrt(np.bincount(np.repeat(np.arange(c.n), np.diff(c.indptr)),
                                  weights=c.val.astype(np.float64) ** 2, minlength=c.n))
        c.val = (c.val / np.repeat(np.where(nrm > 0, nrm, 1), np.diff(c.indptr))).astype(np.float32)
    i, j, s, _ = run_join(aps, c, t, device_input=False)
    compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), max(c.n, 1), csr=c)


def test_dense_dimension_in_every_vector(aps):
    rng = np.random.default_rng(8)
    rows = [{0: 1.0 + rng.random(), int(rng.integers(1, 300)): rng.random() + 0.1} for _ in range(3000)]
    c = csr_raw(rows, 300)
    nrm = np.sqrt(np.add.reduceat(c.val.astype(np.float64) ** 2, c.indptr[:-1]))
    c.val = (c.val / np.repeat(nrm, 2)).astype(np.float32)
    t = 0.9
    i, j, s, _ = run_join(aps, c, t)
    compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), c.n, csr=c)


# ------------------------------------------------------------------- errors


@pytest.mark.parametrize(
    "mutate,msg",
    [
        (lambda c: c.idx.__setitem__(slice(0, 2), c.idx[1::-1].copy()), "increasing"),
        (lambda c: c.val.__setitem__(3, -c.val[3]), "value"),
        (lambda c: c.val.__setitem__(3, np.float32(np.nan)), "value"),
        (lambda c: c.idx.__setitem__(5, c.m + 3), "out of"),
        (lambda c: c.val.__setitem__(slice(int(c.indptr[7]), int(c.indptr[8])), 0.9), "norm"),
    ],
)
def test_malformed_input_is_rejected(aps, mutate, msg):
    import paper_1402_3010_gb300 as A

    c, t = synth.config_small(seed=9, n=100, m=400)
    c.idx = c.idx.copy()
    c.val = c.val.copy()
    # make sure row 0 has two components for the ordering case
    assert c.indptr[1] - c.indptr[0] >= 2 or msg != "increasing"
    mutate(c)
    with pytest.raises(A.APSError) as e:
        A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    assert e.value.status == A.EINVAL
    assert msg in str(e.value)


@pytest.mark.parametrize("t", [0.0, -0.1, 1.5, float("nan")])
def test_threshold_out_of_range(aps, t):
    import paper_1402_3010_gb300 as A

    c, _ = synth.config_small(seed=9, n=50, m=100)
    with pytest.raises(A.APSError) as e:
        A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    assert e.value.status == A.EINVAL


def test_injected_allocation_failure_then_recovery(aps):
    import paper_1402_3010_gb300 as A

    c, t = synth.config_small(seed=10, n=300, m=600)
    A.aps_debug_fail_alloc(3)
    with pytest.raises(A.APSError) as e:
        A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    assert e.value.status == A.ENOMEM
    A.aps_debug_fail_alloc(0)
    i, j, s, _ = run_join(aps, c, t)
    compare(i, j, s, oracle.bruteforce(c, f32(t)), f32(t), c.n, csr=c)


# ------------------------------------------------------------------- index steps


def _split_is_valid(cv, mwr, cr, a, b, k, t):
    """Partial indexing at k: the bound sum x[i]*maxweight_i(V) of the first k components
    stays below t and the next component brings it to t (exact rationals; 1e-12 slack for
    the float64 rounding of the running bound)."""
    from fractions import Fraction

    bound = Fraction(0)
    for p in range(a, a + k):
        bound += Fraction(float(cv[p])) * Fraction(float(mwr[cr[p]]))
    ok = bound < Fraction(t) or abs(float(bound) - t) < 1e-12
    if a + k < b:
        nxt = bound + Fraction(float(cv[a + k])) * Fraction(float(mwr[cr[a + k]]))
        ok = ok and (nxt >= Fraction(t) or abs(float(nxt) - t) < 1e-12)
    return ok


@pytest.mark.parametrize("hi", [300, 64])
def test_index_build_steps_match_oracle(aps, hi):
    """a1 statistics, a2 ranks and rank-ordered rows, a3 partial-indexing split and a4
    posting lists, each against the oracle's step: bit-exact, except that the split (whose
    float64 running bound the GPU sums in another association order) may fall elsewhere
    where the bound comes within rounding of t; there it is checked for validity and
    maximality in exact arithmetic. hi = 64: no row longer than 64 components, so the
    rank-ordered rows come from the in-warp sort instead of the global one."""
    import paper_1402_3010_gb300 as A

    c = pl_small(61, n=4000, m=3000, hi=hi)
    assert np.diff(c.indptr).max() <= 64 if hi == 64 else np.diff(c.indptr).max() > 64
    t = 0.7
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    try:
        ex = A.aps_index_export(h)
    finally:
        A.aps_index_free(h)
    ln, mw, nd, md = oracle.stats(c)
    assert np.array_equal(ex["len"], ln)
    assert np.array_equal(ex["mw"], mw)
    assert np.array_equal(ex["nnz_d"], nd)
    assert np.array_equal(ex["mw_d"], md)
    split, mwp, aux = oracle.prefix_split(c, f32(t))
    assert np.array_equal(ex["rank_of_dim"], aux["rank"])
    assert np.array_equal(ex["crank"], aux["crank"])
    assert np.array_equal(ex["cval"], aux["cval"])
    assert np.array_equal(ex["qsplit"], ex["split"])
    differ = np.nonzero(ex["split"] != split)[0]
    assert differ.size <= max(2, c.n // 1000)
    mwr = aux["mwr"]
    for x in differ.tolist():
        a, b = int(c.indptr[x]), int(c.indptr[x + 1])
        assert _split_is_valid(aux["cval"], mwr, aux["crank"], a, b, int(ex["split"][x]), f32(t))
    split = ex["split"]
    mwp = np.array([aux["cval"][c.indptr[x]:c.indptr[x] + split[x]].max() if split[x] else 0.0 for x in range(c.n)],
                   np.float32)
    assert np.array_equal(ex["mw_pre"], mwp)
    # posting lists: per rank, the multiset of (vector, weight) of the indexed suffixes
    rows = np.repeat(np.arange(c.n), np.diff(c.indptr))
    pos = np.arange(c.nnz) - c.indptr[rows]
    suf = pos >= split[rows]
    ref_r, ref_id, ref_w = aux["crank"][suf], rows[suf], aux["cval"][suf]
    lp = ex["list_ptr"]
    assert lp[-1] == suf.sum()
    got_r = np.repeat(np.arange(c.m), np.diff(lp))
    o1 = np.lexsort((ref_id, ref_r))
    o2 = np.lexsort((ex["post_id"], got_r))
    assert np.array_equal(got_r[o2], ref_r[o1])
    assert np.array_equal(ex["post_id"][o2], ref_id[o1])
    assert np.array_equal(ex["post_w"][o2], ref_w[o1])
    # layout: every list in increasing vector id
    for r in range(0, c.m, 37):
        assert np.all(np.diff(ex["post_id"][lp[r]:lp[r + 1]]) > 0)


def test_queryable_split_uses_norm_bound(aps):
    import paper_1402_3010_gb300 as A

    c = pl_small(62, n=1500, m=1200)
    t = 0.7
    h = A.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t, A.QUERYABLE)
    try:
        ex = A.aps_index_export(h)
    finally:
        A.aps_index_free(h)
    for x in range(0, c.n, 7):
        a, b = c.indptr[x], c.indptr[x + 1]
        k = ex["split"][x]
        pre = ex["cval"][a:a + k].astype(np.float64)
        assert np.sqrt((pre ** 2).sum()) < t
        if a + k < b:
            nxt = ex["cval"][a:a + k + 1].astype(np.float64)
            assert np.sqrt((nxt ** 2).sum()) * np.sqrt(1 + 2e-3) >= t * (1 - 1e-12)


# ------------------------------------------------------------------- batched


def test_batched_instances_match_per_instance_oracle(aps):
    import paper_1402_3010_gb300 as A

    rng = np.random.default_rng(70)
    insts = []
    for k in range(24):
        n = int(np.exp(rng.uniform(np.log(5), np.log(9000))))
        rr = np.random.default_rng([70, k])
        lengths = synth.poisson_lengths(rr, n, 12, 1, 80)
        c = synth.sparse_vectors(n, 3000, lengths, 1.1, "uniform", 0, rng=rr)
        insts.append((c, f32(rng.uniform(0.6, 0.9))))
    insts.append((csr_raw([], 5), 0.7))  # an empty instance in the middle
    insts.append((csr_raw([{1: 1.0}], 5), 0.7))
    args = [(c.indptr, c.idx, c.val, c.n, c.m, t) for c, t in insts]
    outs, st = A.aps_batch_all_pairs(args)
    try:
        total = 0
        for (c, t), p in zip(insts, outs):
            i, j, s = A.pairs_to_numpy(p)
            compare(i, j, s, oracle.bruteforce(c, t), t, max(c.n, 1), csr=c)
            total += len(i)
        assert st["pairs"] == total
        assert st["evaluations"] == sum(c.n * (c.n - 1) // 2 for c, _ in insts)
    finally:
        for p in outs:
            A.aps_pairs_free(p)


def test_batched_concatenated_csr_matches_per_instance_oracle(aps):
    import paper_1402_3010_gb300 as A

    rng = np.random.default_rng(71)
    k = 40
    ns = np.exp(rng.uniform(np.log(3), np.log(12000), size=k)).astype(np.int64)
    ns[5] = 0
    ts = rng.uniform(0.6, 0.9, size=k).astype(np.float32)
    lengths = synth.poisson_lengths(rng, int(ns.sum()), 10, 1, 60)
    c = synth.sparse_vectors(int(ns.sum()), 2000, lengths, 1.1, "uniform", 71, rng=rng)
    ro = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    m = np.full(k, 2000, np.int32)
    import torch

    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    outs, st = A.aps_batch_all_pairs_csr(ro, *dev, m, ts)
    try:
        total = 0
        for r in range(k):
            a, b = int(ro[r]), int(ro[r + 1])
            ip = c.indptr[a:b + 1] - c.indptr[a]
            cr = synth.SparseCSR(ip, c.idx[c.indptr[a]:c.indptr[b]], c.val[c.indptr[a]:c.indptr[b]], b - a, 2000)
            i, j, s = A.pairs_to_numpy(outs[r])
            compare(i, j, s, oracle.bruteforce(cr, float(ts[r])), float(ts[r]), max(b - a, 1), csr=cr)
            total += len(i)
        assert st["pairs"] == total
    finally:
        for o in outs:
            A.aps_pairs_free(o)


@pytest.mark.parametrize("t", [0.5, 0.7, 0.9])
def test_full_size_200k_sampled_rows(aps, t):
    """The 200k x 100k power-law workload at each threshold of its sweep, in the bench's
    configuration (device CSR, default flags): 40 sampled vectors' pairs checked one by one
    against the oracle's float64 brute force over the whole set, plus the global form of
    the result (checked on the device, where the pairs stay)."""
    import torch

    c = synth.config_large()
    t = f32(t)
    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    h = aps.aps_build_index(*dev, c.n, c.m, t)
    try:
        p = aps.aps_all_pairs(h)
        try:
            gi, gj, gs = aps.pairs_to_torch(p)
        finally:
            aps.aps_pairs_free(p)
        st = aps.aps_index_stats(h)
    finally:
        aps.aps_index_free(h)
    assert gi.numel() == st["pairs"] > 1_000_000
    gkeys = gi.long() * c.n + gj.long()
    assert bool((gkeys[1:] > gkeys[:-1]).all()) and bool((gi < gj).all())
    rows = np.random.default_rng(3).choice(c.n, 40, replace=False)
    rt = torch.from_numpy(rows.astype(np.int32)).cuda()
    sel = torch.isin(gi, rt) | torch.isin(gj, rt)
    keys = gkeys[sel].cpu().numpy()
    s = gs[sel].cpu().numpy()
    del gi, gj, gs, gkeys, sel
    ref = oracle.bruteforce_rows(c, t, rows)
    rk = ref.keys(c.n)
    rmap = dict(zip(rk.tolist(), ref.s.tolist()))
    gmap = dict(zip(keys.tolist(), s.tolist()))
    assert len(rmap) > 0
    for k in set(rmap) - set(gmap):  # only pairs inside the 1e-5 band may differ
        assert abs(rmap[k] - t) <= 1e-5
    for k in set(gmap) - set(rmap):  # an extra pair is judged by its float64 score
        assert abs(row_dot64(c, *divmod(k, c.n)) - t) <= 1e-5
    common = set(gmap) & set(rmap)
    assert max(abs(gmap[k] - rmap[k]) for k in common) <= 1e-5


def test_batched_workload_shape_sampled_instances(aps):
    """The batched workload's generator and thresholds (64 of its instances, concatenated
    CSR, one call): 6 sampled instances against the oracle's brute force."""
    import torch

    import paper_1402_3010_gb300 as A

    ro, c, m, ts = synth.config_batched_csr(k=64)
    dev = [torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val)]
    outs, st = A.aps_batch_all_pairs_csr(ro, *dev, m, ts)
    try:
        assert sum(int(o.count) for o in outs) == st["pairs"]
        sizes = np.diff(ro)
        pick = np.argsort(sizes)[[0, 10, 30, 45, 55, 60]]
        for r in pick.tolist():
            a, b = int(ro[r]), int(ro[r + 1])
            ip = c.indptr[a:b + 1] - c.indptr[a]
            cr = synth.SparseCSR(ip, c.idx[c.indptr[a]:c.indptr[b]], c.val[c.indptr[a]:c.indptr[b]], b - a, int(m[r]))
            i, j, s = A.pairs_to_numpy(outs[r])
            compare(i, j, s, oracle.bruteforce(cr, float(ts[r])), float(ts[r]), max(b - a, 1), csr=cr)
    finally:
        for o in outs:
            A.aps_pairs_free(o)
