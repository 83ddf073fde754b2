"""Comparison of a CUDA result with the oracle's pair set (shared by the GPU tests).

Acceptance: pairs sorted by (i, j) with i < j (self-joins), identical pair sets except
pairs whose float64 score lies within `band` of t, and float32 scores within `tol` of
the float64 score. A pair only the CUDA path reports is judged by its float64 score,
recomputed here from the inputs (never by the score the CUDA path returned): the caller
names the inputs with `csr=` (rows of a self-join, or the indexed set of a query result
together with `queries=`) or `dense=` (the rows of a dense self-join)."""
import numpy as np


def row_dot64(c, a, b, q=None):
    """float64 dot product of row a of q (default: of c) with row b of c."""
    ia, va = (q if q is not None else c).row(int(a))
    ib, vb = c.row(int(b))
    common, pa, pb = np.intersect1d(ia, ib, assume_unique=True, return_indices=True)
    return float(np.dot(va[pa].astype(np.float64), vb[pb].astype(np.float64)))


def dense_dot64(X, a, b):
    return float(np.dot(X[int(a)].astype(np.float64), X[int(b)].astype(np.float64)))


def compare(i, j, s, ref, t, n, *, band=1e-5, tol=1e-5, self_join=True, csr=None, queries=None, dense=None):
    if csr is None and dense is None:
        raise ValueError("compare() needs the inputs (csr= or dense=) to recompute extra pairs in float64")
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    s = np.asarray(s, np.float64)
    keys = i * n + j
    assert np.all(np.diff(keys) > 0), "pairs must be strictly increasing in (i, j)"
    if self_join:
        assert np.all(i < j), "self-join pairs must have i < j"
    rk = ref.keys(n)
    gpu_only = np.setdiff1d(keys, rk, assume_unique=True)
    ref_only = np.setdiff1d(rk, keys, assume_unique=True)
    rmap = dict(zip(rk.tolist(), ref.s.tolist()))
    for k in ref_only.tolist():
        assert abs(rmap[k] - t) <= band, f"missing pair {divmod(k, n)} score {rmap[k]} (t={t})"
    for k in gpu_only.tolist():
        a, b = divmod(k, n)
        sc = dense_dot64(dense, a, b) if dense is not None else row_dot64(csr, a, b, queries)
        assert abs(sc - t) <= band, f"extra pair {(a, b)} float64 score {sc} (t={t})"
    common = np.intersect1d(keys, rk, assume_unique=True)
    gi = np.searchsorted(keys, common)
    ri = np.searchsorted(rk, common)
    err = np.abs(s[gi] - ref.s[ri]).max() if common.size else 0.0
    assert err <= tol, f"score error {err} > {tol}"
    return {"pairs": int(keys.size), "ref": int(rk.size), "max_err": float(err),
            "gpu_only": int(gpu_only.size), "ref_only": int(ref_only.size)}


def compare_large(i, j, s, ri, rj, rs, t, n, dot64, *, band=1e-5, tol=1e-5, self_join=True):
    """compare() for large sets, vectorised: (i, j, s) from the CUDA path, (ri, rj, rs) the
    oracle's pairs sorted by (i, j). Pairs only one side has must lie within `band` of t by
    their float64 score (recomputed with dot64(a, b) for the CUDA path's extras); scores of
    the common pairs within `tol` of the oracle's."""
    keys = np.asarray(i, np.int64) * n + np.asarray(j, np.int64)
    rk = np.asarray(ri, np.int64) * n + np.asarray(rj, np.int64)
    assert np.all(keys[1:] > keys[:-1]), "pairs must be strictly increasing in (i, j)"
    if self_join:
        assert np.all(np.asarray(i) < np.asarray(j)), "self-join pairs must have i < j"
    rs = np.asarray(rs, np.float64)
    s = np.asarray(s, np.float64)
    pos = np.searchsorted(rk, keys)
    pos_c = np.minimum(pos, max(rk.size - 1, 0))
    hit = (pos < rk.size) & (rk[pos_c] == keys) if rk.size else np.zeros(keys.size, bool)
    extra = keys[~hit]
    rpos = np.searchsorted(keys, rk)
    rpos_c = np.minimum(rpos, max(keys.size - 1, 0))
    rhit = (rpos < keys.size) & (keys[rpos_c] == rk) if keys.size else np.zeros(rk.size, bool)
    missing = ~rhit
    assert np.all(np.abs(rs[missing] - t) <= band), \
        f"{int(missing.sum())} missing pairs, e.g. {divmod(int(rk[missing][0]), n)} score {rs[missing][0]}"
    for k in extra.tolist():
        a, b = divmod(k, n)
        sc = dot64(a, b)
        assert abs(sc - t) <= band, f"extra pair {(a, b)} float64 score {sc} (t={t})"
    err = float(np.abs(s[hit] - rs[pos_c[hit]]).max()) if hit.any() else 0.0
    assert err <= tol, f"score error {err} > {tol}"
    return {"pairs": int(keys.size), "ref": int(rk.size), "max_err": err, "gpu_only": int(extra.size),
            "ref_only": int(missing.sum())}
