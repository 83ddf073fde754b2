"""The CPU oracle on every host core, for parity checks at full size (test infrastructure).

Worker processes are spawned (never forked: a process forked after CUDA was initialised
can hang) and read their input from files, so that large sets are not pickled.

- all_pairs_parallel: the oracle's sequential all-pairs-2 (Alg. 1-2 with the all-pairs-1/2
  bounds) over one set, with the query vectors dealt round-robin to the workers; every
  worker indexes the whole set and matches its own queries, and the union of the workers'
  pairs is the full pair set (each pair is found once, by its later vector).
- instances_parallel: the same program over many independent instances, one per task.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import tempfile

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_csr(path):
    sys.path.insert(0, _ROOT)
    import synth

    with np.load(path) as z:
        return synth.SparseCSR(z["indptr"], z["idx"], z["val"], int(z["n"]), int(z["m"]))


def _set_worker(job):
    path, t, k, cores, out = job
    sys.path.insert(0, _ROOT)
    import oracle

    c = _load_csr(path)
    mask = (np.arange(c.n) % cores == k).astype(np.uint8)
    pairs, cnt = oracle.all_pairs(c, t, oracle.ALL_PAIRS_2, query_mask=mask)
    np.savez(out, i=pairs.i, j=pairs.j, s=pairs.s)
    return out, cnt["evaluations"]


def all_pairs_parallel(c, t: float, cores: int | None = None):
    """(i, j, s) of every pair i < j with dot >= t, sorted by (i, j), float64 scores."""
    cores = cores or os.cpu_count() or 1
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "set.npz")
        np.savez(path, indptr=c.indptr, idx=c.idx, val=c.val, n=c.n, m=c.m)
        jobs = [(path, float(t), k, cores, os.path.join(d, f"p{k}.npz")) for k in range(cores)]
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_set_worker, jobs)
        parts = [np.load(r[0]) for r in res]
        i = np.concatenate([p["i"] for p in parts]).astype(np.int64)
        j = np.concatenate([p["j"] for p in parts]).astype(np.int64)
        s = np.concatenate([p["s"] for p in parts])
    keys = i * c.n + j
    o = np.argsort(keys, kind="stable")
    return i[o], j[o], s[o]


def _inst_worker(job):
    path, lo, hi, ro, m, ts = job
    sys.path.insert(0, _ROOT)
    import oracle
    import synth

    c = _load_csr(path)
    out = []
    for r in range(lo, hi):
        a, b = int(ro[r]), int(ro[r + 1])
        cr = synth.SparseCSR(c.indptr[a:b + 1] - c.indptr[a], c.idx[c.indptr[a]:c.indptr[b]],
                             c.val[c.indptr[a]:c.indptr[b]], b - a, int(m[r]))
        p, _ = oracle.all_pairs(cr, float(ts[r]), oracle.ALL_PAIRS_2)
        out.append((p.i, p.j, p.s))
    return out


def instances_parallel(ro, c, m, ts, cores: int | None = None):
    """The oracle's pairs of every instance of a concatenated batch (as synth's batched
    configurations return it): a list of (i, j, s) per instance, local ids."""
    cores = cores or os.cpu_count() or 1
    k = len(ro) - 1
    # cut the instances into contiguous runs of about equal evaluations
    w = np.diff(ro).astype(np.float64) ** 2
    cuts = np.searchsorted(np.cumsum(w), np.linspace(0, w.sum(), 4 * cores + 1)[1:-1])
    bounds = np.unique(np.concatenate([[0], np.minimum(cuts + 1, k), [k]]))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "batch.npz")
        np.savez(path, indptr=c.indptr, idx=c.idx, val=c.val, n=c.n, m=c.m)
        jobs = [(path, int(a), int(b), ro, m, ts) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_inst_worker, jobs)
    return [x for part in res for x in part]
