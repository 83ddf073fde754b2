"""The seeded workload generators against the recipes they implement (host only): the
power-law length laws solved for their means, the large sparse set, the dense mixture
under the noise-norm reading, and the batched set."""
import math

import numpy as np

import synth


def _power_law_mean(alpha, lo, hi):
    k = np.arange(lo, hi + 1, dtype=np.float64)
    p = k ** -alpha
    p /= p.sum()
    return float((k * p).sum()), float(p[0])


def test_power_law_exponents_give_their_stated_means():
    """The exponents are solved for mean |x| = 50 on [1, 2000] (large sparse set) and 40
    (serving index); the law itself, not a sample, is checked."""
    mean50, p1 = _power_law_mean(synth.ALPHA_MEAN50, 1, 2000)
    assert abs(mean50 - 50.0) < 0.05
    assert abs(p1 - 0.342) < 0.002  # about a third of the vectors have one component
    mean40, _ = _power_law_mean(synth.ALPHA_MEAN40, 1, 2000)
    assert abs(mean40 - 40.0) < 0.05


def test_large_sparse_set_follows_its_recipe():
    c = synth.config_large()
    assert (c.n, c.m) == (200_000, 100_000)
    ln = np.diff(c.indptr)
    assert ln.min() >= 1 and ln.max() <= 2000
    assert abs(ln.mean() - 50.0) < 1.0
    assert abs((ln == 1).mean() - 0.342) < 0.01
    nd = np.bincount(c.idx, minlength=c.m)
    assert 70_000 < nd.max() < 90_000  # the densest dimension (Zipf(1.0) head)
    for r in range(0, c.n, 9973):
        ids, vals = c.row(r)
        assert np.all(np.diff(ids) > 0) and np.all(vals > 0)
        assert abs(float(np.sum(vals.astype(np.float64) ** 2)) - 1.0) < 1e-5


def test_dense_mixture_uses_the_noise_norm_reading():
    """x = normalize(mu_k + (0.15 / sqrt(d)) z): every row has cluster-mates at cosine
    near 1 / sqrt(1 + 0.15^2) ~ 0.989 (about 0.978 between two noisy members), while
    unrelated rows are near orthogonal; the per-coordinate reading would give none."""
    X, t = synth.config_dense()
    assert X.shape == (200_000, 256) and t == 0.8
    X64 = X.astype(np.float64)
    assert np.abs(np.linalg.norm(X64[::997], axis=1) - 1.0).max() < 1e-6
    rows = np.random.default_rng(9).choice(X.shape[0], 12, replace=False)
    for r in rows.tolist():
        cos = X64 @ X64[r]
        cos[r] = -1.0
        assert cos.max() > 0.95
        assert abs(float(np.median(cos))) < 0.02
        assert 20 < int((cos >= t).sum()) < 400  # about 100 members per component


def test_batched_set_follows_its_recipe():
    ro, c, m, ts = synth.config_batched_csr()
    ns = np.diff(ro)
    assert len(ns) == 512 and np.all(m == 50_000)
    assert ns.min() >= 100 and ns.max() <= 20_000
    # log-uniform sizes: the median is near the geometric mean of the bounds
    assert abs(math.log(float(np.median(ns))) - 0.5 * math.log(100 * 20_000)) < 0.3
    assert ts.min() >= 0.6 and ts.max() <= 0.9
    ln = np.diff(c.indptr)
    assert ln.min() >= 1 and ln.max() <= 300 and abs(ln.mean() - 30.0) < 0.5
