"""2-D (checkerboard) All-Pairs over a q x r mesh of host ranks, after Sec. 6 (Alg. 7,
Par-All-Pairs-0-2D): the horizontal algorithm (Alg. 6) over the mesh's rows and the
vertical one with local pruning (Sec. 5.1, Lemma 1, local threshold t/r) over its columns.

Rank k sits at row a = k // r and column c = k % r. Vectors are dealt cyclically over the q
rows (global id g in row g % q, as the horizontal driver deals them over its ranks), and the
dimensions are binned into r blocks by the vertical algorithm's initial distribution. Rank
(a, c) holds row a's vectors restricted to block c's dimensions. For every row b <= a it
finds the local pairs of the block at the local threshold: b = a by the self-join of its
projection, b < a by matching row b's projected vectors (received from rank (b, c): the
paper's gather along the processor column) against its index. By Lemma 1 a match of rows
(a, b) reaches t/r on at least one block, so the union of row a's r local results holds all
of them; row a's first rank (a, 0) completes that union exactly (duplicates dropped, each
pair's dot product recomputed in float64 from the full rows, kept when >= t), and the
collector concatenates the rows' results in (i, j) order.

Parts and results go through a key-value store (as in the horizontal driver, which also
supplies the store helpers), which carries the failure detection: a completer that waits in
vain for a rank's local pairs recomputes them from the partition, and the collector
recomputes a row whose completed result never arrives. Failures are host-side only; no GPU
kernel waits on another rank and a process uses at most one GPU.
"""
from __future__ import annotations

import numpy as np

from .horizontal import Part, RankFailed, _get, _put, cyclic_part
from .vertical import local_threshold, partition_dims


def mesh_shape(p: int, q: int):
    """(q, r) of a mesh of p ranks with q rows."""
    if q < 1 or p % q:
        raise ValueError(f"{p} ranks do not form a mesh with {q} rows")
    return q, p // q


def block_part(part: Part, block, c: int) -> Part:
    """A row's part restricted to the dimensions of block c (ids and values unchanged)."""
    keep = np.asarray(block)[part.idx] == c
    row = np.repeat(np.arange(part.n, dtype=np.int64), np.diff(part.indptr))
    ip = np.zeros(part.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(row[keep], minlength=part.n), out=ip[1:])
    return Part(ip, part.idx[keep], part.val[keep], part.gids, part.m)


def dimension_blocks(indptr, idx, m: int, r: int) -> np.ndarray:
    """The columns' dimension blocks (the vertical algorithm's initial distribution)."""
    return partition_dims(np.bincount(np.asarray(idx, dtype=np.int64), minlength=m), r)


class GpuMatcher2D:
    """The library's calls for one rank: the local join of a projection and the query of the
    lower rows' projections against it (indexes of sub-unit rows, at the local threshold),
    and the exact completion of a row's union (``aps_pairs_verify``)."""

    def __init__(self, stream=None):
        from . import load

        load()
        self.stream = stream

    def local(self, part: Part, lower: list, t_local: float):
        from . import (QUERYABLE, SUBUNIT_NORMS, aps_all_pairs, aps_build_index, aps_index_free, aps_pairs_free,
                       aps_query, pairs_to_numpy)

        h = aps_build_index(part.indptr, part.idx, part.val, part.n, part.m, t_local, QUERYABLE | SUBUNIT_NORMS,
                            self.stream)
        try:
            r = aps_all_pairs(h)
            try:
                own = pairs_to_numpy(r)
            finally:
                aps_pairs_free(r)
            cross = []
            for q in lower:
                r = aps_query(h, q.indptr, q.idx, q.val, q.n, t_local, SUBUNIT_NORMS)
                try:
                    cross.append(pairs_to_numpy(r))
                finally:
                    aps_pairs_free(r)
        finally:
            aps_index_free(h)
        return own, cross

    def complete(self, ci, cj, rows: Part, t: float):
        """The candidate pairs (ci < cj, local ids of `rows`, duplicates allowed) whose full
        dot product reaches t, as (i, j, score) in (i, j) order, local ids."""
        from . import aps_pairs, aps_pairs_free, aps_pairs_verify, pairs_to_numpy

        ci = np.ascontiguousarray(ci, dtype=np.int32)
        cj = np.ascontiguousarray(cj, dtype=np.int32)
        # a host candidate list (ci, cj stay alive across the call)
        lst = aps_pairs(count=int(ci.size), i=ci.ctypes.data, j=cj.ctypes.data, score=None, on_device=0)
        out, _ = aps_pairs_verify([lst], rows.indptr, rows.idx, rows.val, rows.n, rows.m, t, 0, self.stream)
        try:
            return pairs_to_numpy(out)
        finally:
            aps_pairs_free(out)


def _join_rows(a: Part, b: Part) -> Part:
    """Rows of a then rows of b as one part (the union a completer rescores)."""
    ip = np.concatenate([a.indptr, a.indptr[-1] + b.indptr[1:]])
    return Part(ip, np.concatenate([a.idx, b.idx]), np.concatenate([a.val, b.val]),
                np.concatenate([a.gids, b.gids]), a.m)


def local_share(part: Part, lower: list, t_local: float, matcher):
    """Rank (a, c)'s local pairs in global ids, oriented (min, max): its block's self-join and
    every lower row's block against it, as one array pair (duplicates are impossible here)."""
    own, cross = matcher.local(part, lower, t_local)
    I, J = [part.gids[own[0]]], [part.gids[own[1]]]
    for q, (qi, pj, _) in zip(lower, cross):
        x, y = q.gids[qi], part.gids[pj]
        I.append(np.minimum(x, y))
        J.append(np.maximum(x, y))
    return np.concatenate(I).astype(np.int64), np.concatenate(J).astype(np.int64)


def complete_row(a: int, shares: list, rows_of, t: float, matcher):
    """Row a's pairs: the union of its r local shares completed exactly against the full rows
    of every row b <= a, in global ids (i < j, (i, j) order)."""
    ci = np.concatenate([s[0] for s in shares]) if shares else np.zeros(0, np.int64)
    cj = np.concatenate([s[1] for s in shares]) if shares else np.zeros(0, np.int64)
    rows = rows_of(a)
    for b in range(a):
        rows = _join_rows(rows, rows_of(b))
    pos = np.argsort(rows.gids, kind="stable")  # global id -> local id of `rows`
    li = pos[np.searchsorted(rows.gids, ci, sorter=pos)]
    lj = pos[np.searchsorted(rows.gids, cj, sorter=pos)]
    lo, hi = np.minimum(li, lj), np.maximum(li, lj)
    i, j, s = matcher.complete(lo, hi, rows, t)
    gi, gj = rows.gids[i], rows.gids[j]
    I, J = np.minimum(gi, gj), np.maximum(gi, gj)
    o = np.lexsort((J, I))
    return I[o], J[o], np.asarray(s, dtype=np.float32)[o]


def twod_all_pairs(rank: int, p: int, q: int, store, indptr, idx, val, m: int, t: float, matcher,
                   timeout_s: float = 30.0, collector: int = 0, fail=None):
    """Run rank `rank` of the 2-D all-pairs on a q x (p / q) mesh over the whole set (indptr,
    idx, val; every rank can re-read it, which is what makes a failed rank's work
    recomputable). Returns (i, j, score, failed) on the collector, pairs in (i, j) order and
    failed the ranks whose work was recomputed, and None elsewhere. timeout_s is the wait
    for a projection; the waits for a rank's local pairs and for a row's result are longer
    multiples of it (the work they wait for may itself have waited).

    fail: host-side fault injection for tests, (rank, stage) with stage "before_part" (the
    rank raises before publishing its projection), "before_local" (after publishing it,
    before its local pairs) or "before_row" (a completer raises before publishing its row's
    result)."""
    q, r = mesh_shape(p, q)
    a, c = divmod(rank, r)
    block = dimension_blocks(indptr, idx, m, r)
    tl = local_threshold(t, r)
    rows_of = lambda b: cyclic_part(indptr, idx, val, m, b, q)  # noqa: E731
    proj_of = lambda b, cc: block_part(rows_of(b), block, cc)  # noqa: E731

    def maybe_fail(stage):
        if fail is not None and fail[0] == rank and fail[1] == stage:
            raise RuntimeError(f"injected failure of rank {rank} at {stage}")

    maybe_fail("before_part")
    mine = proj_of(a, c)
    _put(store, f"aps2d/proj/{a}/{c}", mine)
    maybe_fail("before_local")
    lower = []
    for b in range(a):  # the column's lower rows (their projections on block c)
        x = _get(store, f"aps2d/proj/{b}/{c}", timeout_s)
        lower.append(x if x is not None else proj_of(b, c))
    _put(store, f"aps2d/local/{a}/{c}", local_share(mine, lower, tl, matcher))
    failed = []
    # the waits nest: a rank may first wait for up to a missing projections, a completer for
    # up to r missing shares, so each level waits longer than everything below it
    if c == 0:  # row a's completer
        shares = []
        for cc in range(r):
            sh = _get(store, f"aps2d/local/{a}/{cc}", (a + 2) * timeout_s)
            if sh is None:
                failed.append(a * r + cc)
                sh = local_share(proj_of(a, cc), [proj_of(b, cc) for b in range(a)], tl, matcher)
            shares.append(sh)
        maybe_fail("before_row")
        _put(store, f"aps2d/row/{a}", (complete_row(a, shares, rows_of, t, matcher), failed))
    if rank != collector:
        return None
    parts, failed_all = [], []
    for b in range(q):
        got = _get(store, f"aps2d/row/{b}", (q + r + 2) * timeout_s)
        if got is None:  # the row's completer failed: redo the whole row
            failed_all.append(b * r)
            try:
                shares = [local_share(proj_of(b, cc), [proj_of(x, cc) for x in range(b)], tl, matcher)
                          for cc in range(r)]
                got = (complete_row(b, shares, rows_of, t, matcher), [])
            except Exception as e:
                raise RankFailed(f"row {b} delivered no result and could not be recomputed: {e}") from e
        parts.append(got[0])
        failed_all.extend(got[1])
    i = np.concatenate([x[0] for x in parts])
    j = np.concatenate([x[1] for x in parts])
    s = np.concatenate([x[2] for x in parts])
    o = np.lexsort((j, i))
    return i[o].astype(np.int32), j[o].astype(np.int32), s[o], sorted(set(failed_all))
