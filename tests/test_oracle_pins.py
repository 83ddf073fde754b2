"""Pins for the CPU oracle: it is checked against things other than itself -- a library
routine (scipy.sparse FP64 products), closed forms, the paper's printed numbers
(tests/golden/), the paper's cost formula, and brute force on tiny inputs."""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_from_rows(rows, m):
    """rows: list of dict {dim: value}; values are normalised in FP64 then rounded."""
    indptr = [0]
    idx, val = [], []
    for r in rows:
        ks = sorted(r)
        v = np.array([r[k] for k in ks], dtype=np.float64)
        nrm = np.linalg.norm(v) if v.size else 1.0
        idx.extend(ks)
        val.extend((v / nrm).tolist())
        indptr.append(len(idx))
    return synth.SparseCSR(
        indptr=np.array(indptr, dtype=np.int64),
        idx=np.array(idx, dtype=np.int32),
        val=np.array(val, dtype=np.float32),
        n=len(rows),
        m=m,
    )


def csr_raw(rows, m):
    """rows given with exact float32 values, not normalised."""
    indptr = [0]
    idx, val = [], []
    for r in rows:
        for k in sorted(r):
            idx.append(k)
            val.append(r[k])
        indptr.append(len(idx))
    return synth.SparseCSR(
        indptr=np.array(indptr, dtype=np.int64),
        idx=np.array(idx, dtype=np.int32),
        val=np.array(val, dtype=np.float32),
        n=len(rows),
        m=m,
    )


def random_small(seed, n=120, m=60, mean=6, zipf=1.1, weights="uniform"):
    rng = np.random.default_rng(seed)
    lengths = synth.poisson_lengths(rng, n, mean, 0, m)
    return synth.sparse_vectors(n, m, lengths, zipf, weights, seed, rng=rng)


def scipy_pairs(c, t):
    D = sp.csr_matrix((c.val.astype(np.float64), c.idx, c.indptr), shape=(c.n, c.m))
    S = (D @ D.T).tocoo()
    keep = (S.row < S.col) & (S.data >= t)
    return oracle.Pairs(S.row[keep], S.col[keep], S.data[keep])


def assert_same_outside_band(a, b, t, n, band=1e-9, score_tol=1e-12):
    ka, kb = a.keys(n), b.keys(n)
    sa = dict(zip(ka.tolist(), a.s.tolist()))
    sb = dict(zip(kb.tolist(), b.s.tolist()))
    only_a = [k for k in sa if k not in sb and abs(sa[k] - t) > band]
    only_b = [k for k in sb if k not in sa and abs(sb[k] - t) > band]
    assert not only_a and not only_b, (only_a[:5], only_b[:5])
    for k in set(sa) & set(sb):
        assert abs(sa[k] - sb[k]) <= score_tol, (k, sa[k], sb[k])


# --------------------------------------------------------------- brute force pins


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("t", [0.3, 0.6, 0.9])
def test_bruteforce_matches_scipy_product(seed, t):
    c = random_small(seed, weights="lognormal" if seed % 2 else "uniform")
    got = oracle.bruteforce(c, t)
    ref = scipy_pairs(c, t)
    assert_same_outside_band(got, ref, t, c.n)
    assert np.all(got.i < got.j)


def test_bruteforce_closed_forms():
    # duplicate vectors score ||x||^2 = 1 (to float32 rounding of the normalised values)
    c = csr_from_rows([{0: 1.0, 3: 2.0}, {0: 1.0, 3: 2.0}, {5: 1.0}], 8)
    p = oracle.bruteforce(c, 0.5)
    assert len(p) == 1 and (p.i[0], p.j[0]) == (0, 1)
    assert abs(p.s[0] - 1.0) < 1e-6
    # disjoint supports never match, at any threshold
    c = csr_from_rows([{0: 1.0}, {1: 1.0}, {2: 3.0, 4: 1.0}], 8)
    assert len(oracle.bruteforce(c, 1e-9)) == 0
    # single-nonzero vectors of one dimension: the score is the product of the weights (1*1)
    c = csr_raw([{2: 1.0}, {2: 1.0}, {3: 1.0}], 8)
    p = oracle.bruteforce(c, 1.0)
    assert len(p) == 1 and p.s[0] == 1.0
    # one shared dimension: the score is exactly x[d]*y[d] (exact float32 products)
    c = csr_raw([{1: 0.5, 2: 0.75}, {2: 0.5, 7: 0.25}], 8)
    p = oracle.bruteforce(c, 0.375)
    assert len(p) == 1 and p.s[0] == 0.375
    assert len(oracle.bruteforce(c, 0.3750001)) == 0  # ">= t": a tie at t is a match


def test_bruteforce_rows_and_cross_match_scipy():
    c = random_small(11, n=90)
    q = random_small(12, n=17)
    t = 0.4
    rows = [0, 5, 17, 89]
    got = oracle.bruteforce_rows(c, t, rows)
    full = scipy_pairs(c, t)
    sel = np.isin(full.i, rows) | np.isin(full.j, rows)
    ref = oracle.Pairs(full.i[sel], full.j[sel], full.s[sel])
    # each pair of two listed rows appears twice in bruteforce_rows (once per row)
    keys = np.unique(got.keys(c.n))
    assert np.array_equal(keys, np.unique(ref.keys(c.n)))
    Q = sp.csr_matrix((q.val.astype(np.float64), q.idx, q.indptr), shape=(q.n, q.m))
    D = sp.csr_matrix((c.val.astype(np.float64), c.idx, c.indptr), shape=(c.n, c.m))
    S = (Q @ D.T).tocoo()
    k = S.data >= t
    ref = oracle.Pairs(S.row[k], S.col[k], S.data[k])
    got = oracle.bruteforce_cross(q, c, t)
    assert np.array_equal(got.i, ref.i) and np.array_equal(got.j, ref.j)
    assert np.allclose(got.s, ref.s, rtol=0, atol=1e-12)


# ------------------------------------------------- sequential All-Pairs toggle pins

TOGGLES = [oracle.PARTIAL_INDEX, oracle.MINSIZE, oracle.REMSCORE, oracle.UPPERBOUND]
ALL_SUBSETS = [sum(s) for k in range(5) for s in itertools.combinations(TOGGLES, k)]


def adversarial_cases():
    cases = []
    # identical vectors, plus a near-duplicate
    cases.append((csr_from_rows([{0: 1, 1: 2, 2: 3}] * 4 + [{0: 1, 1: 2, 2: 3.01}], 6), 0.99))
    # single-nonzero vectors, many in the same dimension
    cases.append((csr_raw([{d % 3: 1.0} for d in range(12)], 4), 0.5))
    # ties at exactly t: products and sums exact in float32 and float64
    cases.append((csr_raw([{0: 1.0}, {0: 0.5, 1: 0.75}, {0: 0.5, 1: 0.25, 2: 0.75}, {1: 1.0}], 4), 0.5))
    # t = 1: only exact duplicates
    cases.append((csr_raw([{3: 1.0}, {3: 1.0}, {2: 0.6, 3: 0.8}, {2: 0.6, 3: 0.8}], 5), 1.0))
    # empty rows mixed in
    cases.append((csr_from_rows([{}, {0: 1, 1: 1}, {}, {0: 1, 1: 1.1}, {}], 3), 0.9))
    # one dimension present in every vector (dense dimension)
    rng = np.random.default_rng(5)
    rows = [{0: 1.0 + rng.random(), int(rng.integers(1, 30)): rng.random() + 0.1} for _ in range(60)]
    cases.append((csr_from_rows(rows, 30), 0.7))
    return cases


@pytest.mark.parametrize("flags", ALL_SUBSETS)
def test_all_pairs_every_toggle_subset_equals_bruteforce(flags):
    for seed in range(4):
        for t in (0.35, 0.6, 0.85):
            c = random_small(100 + seed, n=150, m=40, mean=5, zipf=1.0,
                             weights="lognormal" if seed % 2 else "uniform")
            got, cnt = oracle.all_pairs(c, t, flags)
            ref = oracle.bruteforce(c, t)
            assert_same_outside_band(got, ref, t, c.n)
            assert cnt["matches"] == len(got)
    for c, t in adversarial_cases():
        got, _ = oracle.all_pairs(c, t, flags)
        ref = oracle.bruteforce(c, t)
        assert_same_outside_band(got, ref, t, c.n)


def test_all_pairs_0_multiplications_equal_cost_formula():
    """Sec. 3.2.3: all-pairs-0 performs sum_d C(|I_d|, 2) multiplications."""
    for seed in range(3):
        c = random_small(200 + seed, n=300, m=50, mean=8)
        _, cnt = oracle.all_pairs(c, 0.5, 0)
        nnz_d = np.bincount(c.idx, minlength=c.m).astype(np.int64)
        assert cnt["visits"] == int((nnz_d * (nnz_d - 1) // 2).sum())
        assert cnt["evaluations"] == c.n * (c.n - 1) // 2


def test_noopt_scores_every_pair_when_a_dimension_is_shared():
    """Table 6: without pruning, a score is kept for all n(n-1)/2 pairs of radikal
    (every pair shares a dimension). Same property on a set sharing dimension 0."""
    with open(os.path.join(GOLDEN, "noopt_scores.txt")) as f:
        n, scores = [int(v) for v in f.read().split("\n")[-2].split()]
    assert n * (n - 1) // 2 == scores
    rng = np.random.default_rng(9)
    rows = [{0: rng.random() + 0.01, int(rng.integers(1, 80)): rng.random()} for _ in range(200)]
    c = csr_from_rows(rows, 80)
    _, cnt = oracle.all_pairs(c, 0.99, 0)
    assert cnt["candidates"] == 200 * 199 // 2


def test_remscore_forward_order_is_caught():
    """The remscore bound is only sound with partial indexing when x's components are
    walked sparsest-dimension first. The planted forward order must lose pairs on some of
    the test inputs -- showing the inputs can tell the orders apart."""
    flags_bad = oracle.PARTIAL_INDEX | oracle.REMSCORE_FORWARD
    lost = 0
    for seed in range(40):
        c = random_small(300 + seed, n=120, m=30, mean=4, zipf=1.0, weights="lognormal")
        for t in (0.4, 0.6):
            bad, _ = oracle.all_pairs(c, t, flags_bad)
            ref = oracle.bruteforce(c, t)
            lost += len(set(ref.keys(c.n).tolist()) - set(bad.keys(c.n).tolist()))
            good, _ = oracle.all_pairs(c, t, oracle.PARTIAL_INDEX | oracle.REMSCORE)
            assert_same_outside_band(good, ref, t, c.n)
    assert lost > 0


def test_pruning_reduces_work_not_results():
    c = random_small(77, n=400, m=80, mean=6, zipf=1.0, weights="lognormal")
    t = 0.6
    p0, c0 = oracle.all_pairs(c, t, 0)
    p2, c2 = oracle.all_pairs(c, t, oracle.ALL_PAIRS_2)
    assert np.array_equal(p0.keys(c.n), p2.keys(c.n))
    assert c2["visits"] < c0["visits"]
    assert c2["candidates"] < c0["candidates"]


# ---------------------------------------------------------- preprocessing pins


def test_stats_match_scipy_reductions():
    c = random_small(21, n=200, m=70)
    ln, mw, nd, md = oracle.stats(c)
    D = sp.csr_matrix((c.val, c.idx, c.indptr), shape=(c.n, c.m))
    assert np.array_equal(ln, D.getnnz(axis=1))
    assert np.array_equal(nd, D.getnnz(axis=0))
    assert np.array_equal(mw, D.max(axis=1).toarray().ravel().astype(np.float32))
    assert np.array_equal(md, D.max(axis=0).toarray().ravel().astype(np.float32))


def test_dim_rank_is_a_stable_sort_by_decreasing_nnz():
    rng = np.random.default_rng(3)
    nd = rng.integers(0, 6, size=500).astype(np.int32)
    rank = oracle.dim_rank(nd)
    order = np.argsort(-nd.astype(np.int64), kind="stable")  # library stable sort
    assert np.array_equal(rank[order], np.arange(nd.size))


def test_prefix_split_bound_and_maximality():
    """Partial indexing keeps x' = the longest rank-ordered prefix whose bound
    sum x[i]*maxweight_i(V) stays below t (checked in exact rational arithmetic)."""
    from fractions import Fraction

    c = random_small(31, n=150, m=40, mean=7, zipf=1.0, weights="lognormal")
    for t in (0.3, 0.7, 0.95):
        split, mwp, aux = oracle.prefix_split(c, t)
        cr, cv, mwr = aux["crank"], aux["cval"], aux["mwr"]
        for x in range(c.n):
            a, b = int(c.indptr[x]), int(c.indptr[x + 1])
            k = int(split[x])
            bound = Fraction(0)
            for p in range(a, a + k):
                bound += Fraction(float(cv[p])) * Fraction(float(mwr[cr[p]]))
            assert bound < Fraction(t) or abs(float(bound) - t) < 1e-12
            if a + k < b:
                nxt = bound + Fraction(float(cv[a + k])) * Fraction(float(mwr[cr[a + k]]))
                assert nxt >= Fraction(t) or abs(float(nxt) - t) < 1e-12
            assert mwp[x] == (cv[a : a + k].max() if k else 0.0)
            assert np.all(np.diff(cr[a:b]) > 0)


# ----------------------------------------------------------------- dense oracle


def test_dense_oracle_matches_sparse_bruteforce():
    X = synth.dense_mixture(300, 16, 20, 0.15, seed=4)
    t = 0.8
    dense = oracle.dense_all_pairs(X, t, block=64)
    rows = [[(d, float(v)) for d, v in enumerate(r)] for r in X]
    c = csr_raw([{d: v for d, v in r} for r in rows], 16)
    ref = oracle.bruteforce(c, t)
    assert_same_outside_band(dense, ref, t, 300, band=1e-12, score_tol=1e-12)
    sub = oracle.dense_rows(X, t, [0, 7, 299])
    full_sel = np.isin(dense.i, [0, 7, 299]) | np.isin(dense.j, [0, 7, 299])
    assert np.array_equal(np.unique(sub.keys(300)), np.unique(dense.keys(300)[full_sel]))


# ------------------------------------------------------------ Table 1 definitions


def _last_digit_unit(text):
    return 10.0 ** -(len(text.split(".")[1])) if "." in text else 1.0


def test_table1_statistics_definitions():
    """The derived columns of Table 1 follow nnz/n, nnz/m and nnz/(n*m). The paper
    truncates some of them and rounds others (radikal 7.86 is printed 7.8, facebook 3.09
    is printed 3.1), so each value must agree to one unit of its last printed digit."""
    with open(os.path.join(GOLDEN, "table1_datasets.txt")) as f:
        lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(lines) == 5
    for name, n, m, nnz, avs, ads, spars in lines:
        n, m, nnz = int(n), int(m), int(nnz)
        c = synth.SparseCSR(indptr=np.array([0, nnz]), idx=np.zeros(0, np.int32),
                            val=np.zeros(0, np.float32), n=n, m=m)
        st = c.stats()
        for key, txt in (("avg_vector_size", avs), ("avg_dim_size", ads)):
            assert abs(st[key] - float(txt)) < _last_digit_unit(txt) + 1e-12, (name, key)
        mant = spars.split(".")[1].lstrip("0")
        unit = float(spars) / float("0." + mant) * 10.0 ** -len(mant) if mant else 1.0
        assert abs(st["sparsity"] - float(spars)) < unit + 1e-15, name


def test_generators_follow_their_recipes():
    c, t = synth.config_small()
    st = c.stats()
    assert st["n"] == 2000 and st["m"] == 5000 and t == 0.7
    assert 19.0 < st["avg_vector_size"] < 21.0
    ln = np.diff(c.indptr)
    assert ln.min() >= 1 and ln.max() <= 200
    for r in range(0, c.n, 97):
        ids, vals = c.row(r)
        assert np.all(np.diff(ids) > 0) and np.all(vals > 0)
        assert abs(float(np.sum(vals.astype(np.float64) ** 2)) - 1.0) < 1e-5
    # Zipf head: the densest dimension holds far more than the average dimension
    nd = np.bincount(c.idx, minlength=c.m)
    assert nd.max() > 20 * st["avg_dim_size"]
