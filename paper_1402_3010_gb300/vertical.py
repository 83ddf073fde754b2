"""Vertical (dimension-partitioned) All-Pairs with local pruning, after Sec. 5.1
(Par-All-Pairs-0-Vert, Lemma 1 and Eq. 2).

The dimensions are split into p blocks; the join of each block's projection of the
vectors (the vectors restricted to that block's dimensions) at the local threshold
t_local = t/p yields every pair whose partial score on the block reaches t/p. By Lemma 1 a
pair with x.y >= t reaches t/p on at least one block, so the union of the p local results
holds every match; the union is then completed exactly (``aps_pairs_verify``: duplicates
removed, each pair's full dot product recomputed from the rows in float64, kept when
>= t). The p block joins and the merge run on the GPU; the dimension partition and the
projections are host-side data distribution, as in the paper, where they precede the
timed algorithm.

Dimensions are binned as in the paper's initial distribution (Sec. 5.1.1): by decreasing
number of non-zeros, each into the least loaded block, with the per-dimension work
|I_d|(|I_d| + 1)/2 as its load.
"""
from __future__ import annotations

import numpy as np


def partition_dims(nnz_d, p: int) -> np.ndarray:
    """block[d] in [0, p): first-fit of the dimensions, densest first (ties by smaller id),
    each into the block with the least accumulated |I_d|(|I_d| + 1)/2."""
    nnz_d = np.asarray(nnz_d, dtype=np.int64)
    m = nnz_d.size
    order = np.lexsort((np.arange(m), -nnz_d))
    w = nnz_d * (nnz_d + 1) // 2
    load = np.zeros(p, dtype=np.int64)
    block = np.empty(m, dtype=np.int32)
    for d in order:
        k = int(np.argmin(load))
        block[d] = k
        load[k] += w[d]
    return block


def project(indptr, idx, val, block, k: int):
    """The rows restricted to the dimensions of block k (ids and values unchanged)."""
    indptr = np.asarray(indptr, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int32)
    val = np.asarray(val, dtype=np.float32)
    n = indptr.size - 1
    keep = np.asarray(block)[idx] == k
    row = np.repeat(np.arange(n, dtype=np.int64), np.diff(indptr))
    ip = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(row[keep], minlength=n), out=ip[1:])
    return ip, idx[keep], val[keep]


def local_threshold(t: float, p: int) -> float:
    """t/p (Eq. 2), lowered by a relative 1e-6 and rounded down to float32, so that the
    float rounding of the local scores can never hide a block that reaches t/p."""
    tl = np.float32(t / p * (1.0 - 1e-6))
    if float(tl) > t / p * (1.0 - 1e-6):
        tl = np.nextafter(tl, np.float32(0))
    return float(tl)


def vertical_all_pairs(indptr, idx, val, n: int, m: int, t: float, p: int, stream=None):
    """All pairs with x.y >= t through p dimension blocks with local pruning. Returns
    (aps_pairs in (i, j) order, info) with info = {blocks, t_local, local_pairs, candidates};
    free the pairs with aps_pairs_free."""
    from . import SUBUNIT_NORMS, aps_all_pairs, aps_build_index, aps_index_free, aps_pairs_free, aps_pairs_verify

    indptr = np.asarray(indptr, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int32)
    val = np.asarray(val, dtype=np.float32)
    nnz_d = np.bincount(idx, minlength=m)
    block = partition_dims(nnz_d, p)
    tl = local_threshold(t, p)
    lists, local = [], []
    try:
        for k in range(p):
            ip, ix, vv = project(indptr, idx, val, block, k)
            h = aps_build_index(ip, ix, vv, n, m, tl, SUBUNIT_NORMS, stream)
            try:
                r = aps_all_pairs(h)
            finally:
                aps_index_free(h)
            lists.append(r)
            local.append(int(r.count))
        out, nc = aps_pairs_verify(lists, indptr, idx, val, n, m, t, 0, stream)
    finally:
        for r in lists:
            aps_pairs_free(r)
    return out, {"blocks": p, "t_local": tl, "local_pairs": local, "candidates": nc}
