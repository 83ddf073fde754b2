"""Seeded synthetic inputs for the All-Pairs similarity join.

This module is shared by the CPU oracle tests and the CUDA path tests/bench. It only
draws random inputs; it holds none of the join's arithmetic. Every generator is
deterministic for a given seed (NumPy PCG64).

The paper's own datasets (radikal, 20-newsgroups, wikipedia, facebook, virginia-tech;
Sec. 7, Table 1) are not available, so these shapes stand in for them. They keep the
property the paper stresses (Sec. 7.3): dimension density follows a power law, so a
few dense dimensions dominate the work of the inverted-index join.

Sparse matrices are returned as CSR in canonical input form: int64 ``indptr[n+1]``,
int32 ``idx[nnz]`` strictly increasing inside each row, float32 ``val[nnz] > 0``, each
row L2-normalised (norm computed in float64, then rounded to float32).
"""
from __future__ import annotations

import dataclasses
import math
import os
import tempfile

import numpy as np

__all__ = [
    "SparseCSR",
    "bounded_zipf_cdf",
    "sparse_vectors",
    "config_small",
    "config_large",
    "config_dense",
    "config_batched",
    "config_batched_matches",
    "config_serving",
    "dense_mixture",
    "power_law_lengths",
    "serving_queries",
    "serving_arrivals",
    "poisson_lengths",
]


@dataclasses.dataclass
class SparseCSR:
    indptr: np.ndarray  # int64 [n+1]
    idx: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float32 [nnz]
    n: int
    m: int

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def row(self, r: int):
        a, b = int(self.indptr[r]), int(self.indptr[r + 1])
        return self.idx[a:b], self.val[a:b]

    def stats(self) -> dict:
        """Dataset statistics with the definitions of Table 1 (Sec. 7):
        average vector size = nnz/n, average dimension size = nnz/m,
        sparsity = nnz/(n*m)."""
        nnz = self.nnz
        return {
            "n": self.n,
            "m": self.m,
            "nnz": nnz,
            "avg_vector_size": nnz / max(self.n, 1),
            "avg_dim_size": nnz / max(self.m, 1),
            "sparsity": nnz / max(self.n * self.m, 1),
        }


def bounded_zipf_cdf(m: int, s: float) -> np.ndarray:
    """CDF of a Zipf law on ranks 1..m: p(r) proportional to r**-s."""
    w = np.arange(1, m + 1, dtype=np.float64) ** (-float(s))
    c = np.cumsum(w)
    return c / c[-1]


def poisson_lengths(rng, n, mean, lo, hi):
    return np.clip(rng.poisson(mean, size=n), lo, hi).astype(np.int64)


def power_law_lengths(rng, n, alpha, lo, hi):
    """Discrete power law p(k) proportional to k**-alpha on [lo, hi]."""
    k = np.arange(lo, hi + 1, dtype=np.float64)
    c = np.cumsum(k ** (-alpha))
    c /= c[-1]
    u = rng.random(n)
    return (lo + np.searchsorted(c, u, side="left")).astype(np.int64)


def _distinct_zipf_rows(rng, lengths, m, s, chunk=262144):
    """For each row draw bounded-Zipf ranks (0-based) until ``lengths[r]`` distinct ranks
    are collected, i.e. sampling without replacement in draw order. Rows are drawn in
    chunks of ``chunk`` rows (keeps the sort keys within 63 bits)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    if lengths.size > chunk:
        rows, ranks = [], []
        for a in range(0, lengths.size, chunk):
            r, k = _distinct_zipf_rows_chunk(rng, lengths[a : a + chunk], m, s)
            rows.append(r + a)
            ranks.append(k)
        return np.concatenate(rows), np.concatenate(ranks)
    return _distinct_zipf_rows_chunk(rng, lengths, m, s)


def _distinct_zipf_rows_chunk(rng, lengths, m, s):
    n = len(lengths)
    lengths = np.asarray(lengths, dtype=np.int64)
    if np.any(lengths > m):
        raise ValueError("row length exceeds the number of dimensions")
    cdf = bounded_zipf_cdf(m, s)
    rbits = max(1, int(m - 1).bit_length())
    acc_row = np.zeros(0, dtype=np.int64)
    acc_rank = np.zeros(0, dtype=np.int64)
    acc_ord = np.zeros(0, dtype=np.int64)
    done_row, done_rank, done_ord = [], [], []  # rows that already hold all their ranks
    frozen = np.zeros(n, dtype=bool)
    have = np.zeros(n, dtype=np.int64)
    draw_base = 0
    for _round in range(64):
        need = lengths - have
        todo = np.nonzero(need > 0)[0]
        if todo.size == 0:
            break
        # oversample: duplicates are frequent for the head ranks of a Zipf law
        k = (need[todo] * 1.5 + 8).astype(np.int64)
        rows = np.repeat(todo, k)
        ranks = np.searchsorted(cdf, rng.random(rows.size), side="left").astype(np.int64)
        ranks = np.minimum(ranks, m - 1)
        order = draw_base + np.arange(rows.size, dtype=np.int64)
        draw_base += rows.size
        all_row = np.concatenate([acc_row, rows])
        all_rank = np.concatenate([acc_rank, ranks])
        all_ord = np.concatenate([acc_ord, order])
        obits = max(1, int(draw_base).bit_length())
        if all_row.size and int(all_row.max()).bit_length() + rbits + obits > 63:
            raise ValueError("generator keys overflow int64")
        # first occurrence of every (row, rank) in draw order: sort by (row, rank, order)
        key = (((all_row << rbits) | all_rank) << obits) | all_ord
        key.sort()
        rr = key >> obits
        first = np.ones(key.size, dtype=bool)
        first[1:] = rr[1:] != rr[:-1]
        key = key[first]
        r_k = key >> (obits + rbits)
        k_k = (key >> obits) & ((1 << rbits) - 1)
        o_k = key & ((1 << obits) - 1)
        # keep the first lengths[r] distinct ranks of each row, by draw order
        key2 = (r_k << obits) | o_k
        srt = np.argsort(key2, kind="stable")
        r_k, k_k, o_k = r_k[srt], k_k[srt], o_k[srt]
        starts = np.searchsorted(r_k, np.arange(n), side="left")
        pos = np.arange(r_k.size) - starts[r_k]
        sel = pos < lengths[r_k]
        r_k, k_k, o_k = r_k[sel], k_k[sel], o_k[sel]
        got = np.bincount(r_k, minlength=n).astype(np.int64)
        # rows that are complete leave the working set (their selection is final)
        fin = got[r_k] == lengths[r_k]
        done_row.append(r_k[fin])
        done_rank.append(k_k[fin])
        done_ord.append(o_k[fin])
        acc_row, acc_rank, acc_ord = r_k[~fin], k_k[~fin], o_k[~fin]
        frozen[r_k[fin]] = True
        have = np.where(frozen, lengths, got)
    else:  # pragma: no cover - 64 rounds always suffice for the shapes used here
        raise RuntimeError("distinct Zipf sampling did not converge")
    out_row = np.concatenate(done_row + [acc_row])
    out_rank = np.concatenate(done_rank + [acc_rank])
    out_ord = np.concatenate(done_ord + [acc_ord])
    o = np.lexsort((out_ord, out_row))  # by row, then draw order
    return out_row[o], out_rank[o]


def sparse_vectors(
    n: int,
    m: int,
    lengths: np.ndarray,
    zipf_s: float,
    weights: str,
    seed: int,
    rng=None,
    perm=None,
) -> SparseCSR:
    """n sparse non-negative vectors over m dimensions.

    ``lengths[r]`` distinct feature ids per row, drawn from a bounded Zipf(s) law over
    ranks, with ranks mapped to ids through a seeded random permutation of [0, m).
    ``weights`` is ``"uniform"`` (U(0,1], drawn as 1 - U[0,1)) or ``"lognormal"``
    (log-normal, mu=0, sigma=1). Each row is then L2-normalised. A caller-given ``perm``
    (rank -> id) lets two vector sets share their dense dimensions."""
    rng = np.random.default_rng(seed) if rng is None else rng
    rows, ranks = _distinct_zipf_rows(rng, lengths, m, zipf_s)
    if perm is None:
        perm = rng.permutation(m)
    perm = np.asarray(perm, dtype=np.int64)
    ids = perm[ranks]
    if weights == "uniform":
        w = 1.0 - rng.random(rows.size)
    elif weights == "lognormal":
        w = rng.lognormal(0.0, 1.0, size=rows.size)
    else:
        raise ValueError(weights)
    o = np.argsort((rows << 32) | ids, kind="stable")
    rows, ids, w = rows[o], ids[o], w[o]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=indptr[1:])
    norm2 = np.bincount(rows, weights=w * w, minlength=n)
    nrm = np.sqrt(norm2)
    nrm[nrm == 0] = 1.0
    val = (w / nrm[rows]).astype(np.float32)
    return SparseCSR(indptr=indptr, idx=ids.astype(np.int32), val=val, n=n, m=m)


# --- the five workload shapes -------------------------------------------------------


def config_small(seed: int = 1, n: int = 2000, m: int = 5000) -> tuple[SparseCSR, float]:
    """Plain sparse all-pairs: n=2000, m=5000, |x| ~ Poisson(20) clipped to [1,200],
    Zipf(1.1) feature ids, U(0,1] weights, L2-normalised, t=0.7."""
    rng = np.random.default_rng(seed)
    lengths = poisson_lengths(rng, n, 20, 1, min(200, m))
    return sparse_vectors(n, m, lengths, 1.1, "uniform", seed, rng=rng), 0.7


# power-law exponents that give mean 50 (n=200k config) and mean 40 (serving index) on [1,2000]
ALPHA_MEAN50 = 1.4135
ALPHA_MEAN40 = 1.4647


CACHE_DIR = os.environ.get("APS_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "aps-synth-cache"))


def _cached(name: str, make):
    """Reuse a generated CSR across processes of one machine (files under CACHE_DIR)."""
    path = os.path.join(CACHE_DIR, name + ".npz")
    try:
        with np.load(path) as z:
            return SparseCSR(z["indptr"], z["idx"], z["val"], int(z["n"]), int(z["m"]))
    except Exception:
        pass
    c = make()
    try:
        os.makedirs(CACHE_DIR, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, indptr=c.indptr, idx=c.idx, val=c.val, n=c.n, m=c.m)
        os.replace(tmp, path)
    except OSError:
        pass
    return c


def config_large(seed: int = 2, n: int = 200_000, m: int = 100_000) -> SparseCSR:
    """Large sparse all-pairs: n=200k, m=100k, |x| power law on [1,2000] with mean ~50
    (alpha=1.4135), Zipf(1.0) ids, log-normal(0,1) weights, L2-normalised.
    Thresholds swept over {0.5, 0.7, 0.9}."""

    def make():
        rng = np.random.default_rng(seed)
        lengths = power_law_lengths(rng, n, ALPHA_MEAN50, 1, min(2000, m))
        return sparse_vectors(n, m, lengths, 1.0, "lognormal", seed, rng=rng)

    return _cached(f"large-v2-s{seed}-n{n}-m{m}", make)


def dense_mixture(n: int, d: int, k: int, noise_norm: float, seed: int) -> np.ndarray:
    """n unit vectors in R^d from an equal-weight k-component mixture: centre mu_c uniform
    on the unit sphere, x = normalize(mu_c + (noise_norm/sqrt(d)) * z), z ~ N(0, I).
    Returns float32 [n, d], rows normalised in float64 then rounded."""
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal((k, d))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    comp = rng.integers(0, k, size=n)
    out = np.empty((n, d), dtype=np.float32)
    step = 65536
    for a in range(0, n, step):
        b = min(n, a + step)
        x = mu[comp[a:b]] + (noise_norm / math.sqrt(d)) * rng.standard_normal((b - a, d))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[a:b] = x.astype(np.float32)
    return out


def config_dense(seed: int = 3, n: int = 200_000, d: int = 256, k: int = 2000) -> tuple[np.ndarray, float]:
    """Dense embeddings: n=200k, d=256, 2000-component Gaussian mixture with noise norm
    0.15 per vector, L2-normalised, t=0.8."""
    return dense_mixture(n, d, k, 0.15, seed), 0.8


def config_batched(seed: int = 4, k: int = 512, n_lo: int = 100, n_hi: int = 20000, m: int = 50_000):
    """Batched: k independent instances, n log-uniform in [n_lo, n_hi], m=50k, |x| ~
    Poisson(30) clipped to [1,300], Zipf(1.1) ids, U(0,1] weights, t ~ U(0.6, 0.9).
    Returns a list of (SparseCSR, t)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=k)).astype(np.int64)
    ts = rng.uniform(0.6, 0.9, size=k)
    out = []
    for i in range(k):
        sub = np.random.default_rng([seed, i])
        lengths = poisson_lengths(sub, int(ns[i]), 30, 1, 300)
        out.append((sparse_vectors(int(ns[i]), m, lengths, 1.1, "uniform", 0, rng=sub), float(np.float32(ts[i]))))
    return out


def config_batched_csr(seed: int = 4, k: int = 512, n_lo: int = 100, n_hi: int = 20000, m: int = 50_000):
    """The batched workload as one concatenated CSR: instance r owns rows
    [row_offsets[r], row_offsets[r+1]); n log-uniform in [n_lo, n_hi], |x| ~ Poisson(30)
    clipped to [1,300], Zipf(1.1) ids (one rank -> id permutation shared by the instances;
    dimension ids are local to each instance), U(0,1] weights, L2-normalised;
    t ~ U(0.6, 0.9) rounded to float32. Returns (row_offsets, SparseCSR, m[k], t[k])."""

    def make():
        rng = np.random.default_rng(seed)
        ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=k)).astype(np.int64)
        ts = rng.uniform(0.6, 0.9, size=k).astype(np.float32)
        N = int(ns.sum())
        lengths = poisson_lengths(rng, N, 30, 1, 300)
        c = sparse_vectors(N, m, lengths, 1.1, "uniform", seed, rng=rng)
        ro = np.zeros(k + 1, dtype=np.int64)
        np.cumsum(ns, out=ro[1:])
        return SparseCSR(np.concatenate([c.indptr, ro, ts.view(np.int32).astype(np.int64)]), c.idx, c.val, N, m)

    z = _cached(f"batched-v1-s{seed}-k{k}-{n_lo}-{n_hi}-m{m}", make)
    N = z.n
    indptr = z.indptr[: N + 1]
    ro = z.indptr[N + 1 : N + 2 + k]
    ts = z.indptr[N + 2 + k :].astype(np.int32).view(np.float32)
    c = SparseCSR(indptr, z.idx, z.val, N, m)
    return ro, c, np.full(k, m, dtype=np.int32), ts


def config_batched_matches(seed: int = 6, k: int = 512, n_lo: int = 100, n_hi: int = 20000, m: int = 50_000):
    """A second batched set, one that yields matches: the same instance sizes (n log-uniform
    in [n_lo, n_hi]) and thresholds t ~ U(0.6, 0.9), but vectors from the large set's family
    (|x| power law with mean ~50 on [1, 300], Zipf(1.0) ids, log-normal(0,1) weights), so
    that many vectors share their dominant dimensions. Same return form as
    config_batched_csr: (row_offsets, SparseCSR, m[k], t[k])."""

    def make():
        rng = np.random.default_rng(seed)
        ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=k)).astype(np.int64)
        ts = rng.uniform(0.6, 0.9, size=k).astype(np.float32)
        N = int(ns.sum())
        lengths = power_law_lengths(rng, N, ALPHA_MEAN50, 1, 300)
        c = sparse_vectors(N, m, lengths, 1.0, "lognormal", seed, rng=rng)
        ro = np.zeros(k + 1, dtype=np.int64)
        np.cumsum(ns, out=ro[1:])
        return SparseCSR(np.concatenate([c.indptr, ro, ts.view(np.int32).astype(np.int64)]), c.idx, c.val, N, m)

    z = _cached(f"batchedm-v1-s{seed}-k{k}-{n_lo}-{n_hi}-m{m}", make)
    N = z.n
    indptr = z.indptr[: N + 1]
    ro = z.indptr[N + 1 : N + 2 + k]
    ts = z.indptr[N + 2 + k :].astype(np.int32).view(np.float32)
    c = SparseCSR(indptr, z.idx, z.val, N, m)
    return ro, c, np.full(k, m, dtype=np.int32), ts


def _serving_perm(seed: int, m: int) -> np.ndarray:
    return np.random.default_rng([seed, 7919]).permutation(m)


def config_serving(seed: int = 5, n: int = 1_000_000, m: int = 200_000):
    """Serving index: n=1M, m=200k, |x| power law on [1,2000] with mean ~40 (alpha=1.4647),
    Zipf(1.0) ids, log-normal(0,1) weights, L2-normalised; t=0.75."""
    rng = np.random.default_rng(seed)
    lengths = power_law_lengths(rng, n, ALPHA_MEAN40, 1, min(2000, m))

    def make():
        return sparse_vectors(n, m, lengths, 1.0, "lognormal", seed, rng=rng, perm=_serving_perm(seed, m))

    return _cached(f"serving-v1-s{seed}-n{n}-m{m}", make), 0.75


def serving_queries(nq: int, index_seed: int = 5, m: int = 200_000, qseed: int = 55) -> SparseCSR:
    """Query vectors from the serving index's distribution, drawn with their own seed but
    through the index's rank->id permutation, so queries hit the same dense dimensions."""
    rng = np.random.default_rng(qseed)
    lengths = power_law_lengths(rng, nq, ALPHA_MEAN40, 1, min(2000, m))
    return sparse_vectors(nq, m, lengths, 1.0, "lognormal", qseed, rng=rng, perm=_serving_perm(index_seed, m))


def serving_arrivals(num_batches: int, rate_per_s: float, seed: int = 56):
    """Poisson arrival times (seconds) and batch sizes log-uniform in [1, 4096]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=num_batches)
    sizes = np.exp(rng.uniform(0.0, math.log(4096.0), size=num_batches)).astype(np.int64)
    return np.cumsum(gaps), np.clip(sizes, 1, 4096)


def pair_list(n: int, count: int, seed: int, skew: float = 0.0, w_lo: float = 0.5):
    """A seeded pair list in the form the join returns: unique (i < j) pairs strictly
    increasing in (i, j), float32 weights U[w_lo, 1). Endpoints are drawn with probability
    ~ (rank + 1)^-skew over a random vertex permutation (skew 0: uniform; larger: hubs).
    Up to `count` pairs (duplicates and self-pairs are dropped)."""
    rng = np.random.default_rng(seed)
    if n < 2 or count <= 0:
        e = np.zeros(0, dtype=np.int32)
        return e, e.copy(), np.zeros(0, dtype=np.float32)
    p = (np.arange(n, dtype=np.float64) + 1.0) ** (-skew)
    p /= p.sum()
    perm = rng.permutation(n)
    a = perm[rng.choice(n, size=count, p=p)]
    b = perm[rng.choice(n, size=count, p=p)]
    keep = a != b
    lo = np.minimum(a[keep], b[keep]).astype(np.int64)
    hi = np.maximum(a[keep], b[keep]).astype(np.int64)
    key = np.unique(lo * n + hi)
    i = (key // n).astype(np.int32)
    j = (key % n).astype(np.int32)
    s = rng.uniform(w_lo, 1.0, size=key.size).astype(np.float32)
    return i, j, s

