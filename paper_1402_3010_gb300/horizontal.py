"""Horizontal (vector-partitioned) All-Pairs over host ranks, after the outer-loop
parallelisation of Sec. 5.2 (Alg. 6, Par-All-Pairs-0-Horiz).

Every vector has a home rank (cyclic: global id g lives on rank g % p as local id g // p).
Each rank indexes only its own vectors, receives the other ranks' vectors, and matches
the vectors of every lower rank against its local index; together with each rank's
self-join of its own part this finds every pair exactly once (a pair inside part b on
rank b, a pair across parts a < b on rank b), which is the role of the paper's common
processing order. The paper moves size(V)·(p-1) vector elements for the exchange; so does
this driver (each rank reads every lower rank's part).

Ranks exchange parts and results through a key-value store (``torch.distributed.TCPStore``
or anything with ``set``/``get``/``wait``; values are pickled, so the store must be private
to the job's own processes), which also carries failure detection: the
collecting rank waits for each rank's result with a timeout; a rank that never delivers
is declared failed, and its share is recomputed by the collector from the partition
(re-read through ``part_of``). Failures are host-side only (an exception or an exit
between steps); no GPU kernel waits on another rank and nothing here shards a kernel
across GPUs. A process uses at most one GPU (the matcher's).
"""
from __future__ import annotations

import pickle
from dataclasses import dataclass
from datetime import timedelta

import numpy as np


@dataclass
class Part:
    """A rank's vectors as a CSR over the full dimension space, with their global ids."""

    indptr: np.ndarray  # int64 [n_local + 1]
    idx: np.ndarray     # int32
    val: np.ndarray     # float32
    gids: np.ndarray    # int64 [n_local]
    m: int

    @property
    def n(self) -> int:
        return int(self.gids.size)


def cyclic_part(indptr, idx, val, m: int, rank: int, p: int) -> Part:
    """Rows rank, rank + p, rank + 2p, ... of a CSR (the cyclic home assignment)."""
    indptr = np.asarray(indptr, dtype=np.int64)
    n = indptr.size - 1
    gids = np.arange(rank, n, p, dtype=np.int64)
    lens = indptr[gids + 1] - indptr[gids]
    ip = np.zeros(gids.size + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    take = np.concatenate([np.arange(indptr[g], indptr[g + 1]) for g in gids]) if gids.size else np.zeros(0, np.int64)
    return Part(ip, np.asarray(idx, dtype=np.int32)[take], np.asarray(val, dtype=np.float32)[take], gids, int(m))


class GpuMatcher:
    """The library's join (``aps_all_pairs`` on a queryable index of the part) and query
    path (``aps_query`` of another part against it)."""

    def __init__(self, stream=None):
        from . import load

        load()
        self.stream = stream

    def self_and_cross(self, part: Part, lower: list, t: float):
        """Pairs inside `part` (local ids, i < j) and, for each part in `lower`, the pairs
        (query local id, part local id) of its vectors against `part`."""
        from . import (QUERYABLE, aps_all_pairs, aps_build_index, aps_index_free, aps_pairs_free, aps_query,
                       pairs_to_numpy)

        h = aps_build_index(part.indptr, part.idx, part.val, part.n, part.m, t, QUERYABLE, self.stream)
        try:
            r = aps_all_pairs(h)
            try:
                own = pairs_to_numpy(r)
            finally:
                aps_pairs_free(r)
            cross = []
            for q in lower:
                r = aps_query(h, q.indptr, q.idx, q.val, q.n, t)
                try:
                    cross.append(pairs_to_numpy(r))
                finally:
                    aps_pairs_free(r)
        finally:
            aps_index_free(h)
        return own, cross


class RankFailed(RuntimeError):
    """A rank's share could not be obtained or recomputed."""


def _to_global(part: Part, own, cross, lower: list):
    I, J, S = [], [], []
    i, j, s = own
    I.append(part.gids[i])
    J.append(part.gids[j])
    S.append(s)
    for q, (qi, pj, s) in zip(lower, cross):
        a, b = q.gids[qi], part.gids[pj]
        I.append(np.minimum(a, b))
        J.append(np.maximum(a, b))
        S.append(s)
    return np.concatenate(I), np.concatenate(J), np.concatenate(S).astype(np.float32)


PIECE = 4 << 20  # bytes per store value (stores cap a single value's size)


def _put(store, key: str, obj) -> None:
    """Publish obj under key in pieces; the piece count is written last, so a reader that
    sees it finds every piece."""
    b = pickle.dumps(obj)
    n = max(1, (len(b) + PIECE - 1) // PIECE)
    for k in range(n):
        store.set(f"{key}/{k}", b[k * PIECE:(k + 1) * PIECE])
    store.set(f"{key}/n", str(n))


def _get(store, key: str, timeout_s: float):
    """The object published under key, or None if it does not appear within timeout_s."""
    try:
        store.wait([f"{key}/n"], timedelta(seconds=timeout_s))
    except Exception:
        return None
    n = int(store.get(f"{key}/n"))
    return pickle.loads(b"".join(store.get(f"{key}/{k}") for k in range(n)))


def rank_share(part: Part, lower: list, t: float, matcher):
    """The pairs rank b owns: its part's self-join and every lower part against it,
    in global ids, oriented (min, max)."""
    own, cross = matcher.self_and_cross(part, lower, t)
    return _to_global(part, own, cross, lower)


def horizontal_all_pairs(rank: int, p: int, store, part_of, t: float, matcher, timeout_s: float = 30.0,
                         collector: int = 0, fail=None):
    """Run one rank of the horizontal all-pairs. part_of(r) returns rank r's Part (a rank
    calls it for itself; the collector also calls it to recompute a failed rank's share).
    Returns (i, j, score, failed_ranks) on the collector, pairs in (i, j) order, and None
    elsewhere.

    fail: host-side fault injection for tests, (rank, stage) with stage "before_part" (the
    rank raises before publishing its vectors) or "before_result" (after publishing them,
    before its result); it only affects that rank."""
    def maybe_fail(stage):
        if fail is not None and fail[0] == rank and fail[1] == stage:
            raise RuntimeError(f"injected failure of rank {rank} at {stage}")

    maybe_fail("before_part")
    part = part_of(rank)
    _put(store, f"aps/part/{rank}", part)
    maybe_fail("before_result")
    lower = []
    for a in range(rank):
        q = _get(store, f"aps/part/{a}", timeout_s)
        if q is None:
            q = part_of(a)  # the lower rank never published: re-read its partition
        lower.append(q)
    share = rank_share(part, lower, t, matcher)
    _put(store, f"aps/pairs/{rank}", share)
    if rank != collector:
        return None
    shares, failed = [], []
    for b in range(p):
        sh = _get(store, f"aps/pairs/{b}", timeout_s)
        if sh is None:
            failed.append(b)
            try:
                pb = part_of(b)
                lb = [part_of(a) for a in range(b)]
            except Exception as e:  # the partition cannot be re-read
                raise RankFailed(f"rank {b} delivered no result and its partition cannot be re-read: {e}") from e
            sh = rank_share(pb, lb, t, matcher)
        shares.append(sh)
    i = np.concatenate([x[0] for x in shares])
    j = np.concatenate([x[1] for x in shares])
    s = np.concatenate([x[2] for x in shares])
    order = np.lexsort((j, i))
    return i[order].astype(np.int32), j[order].astype(np.int32), s[order], failed
