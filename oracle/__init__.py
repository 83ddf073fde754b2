"""CPU oracle for the All-Pairs similarity join -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg (and its
``--impl reference`` arm) may import this package. The product path
(``paper_1402_3010_gb300``) never imports it and shares no code with it.

The sparse oracle is plain C (``aps_oracle.c``, FP64, compiled with gcc on first use or by
``__graft_entry__.build()``); this module only marshals arguments. The dense oracle is
NumPy FP64 ``X @ X.T`` followed by the threshold, i.e. the matrix view S = D.D^T of
Sec. 2.1 evaluated by a library routine.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  bruteforce           pinned to scipy.sparse FP64 D.D^T + threshold, closed forms
  all_pairs (toggles)  pinned to bruteforce on tiny random/adversarial inputs, and the
                       all-pairs-0 multiplication count to sum_d C(|I_d|,2) (Sec. 3.2.3)
  stats / dim_rank /
  prefix_split         pinned to NumPy restatements of their definitions and to the
                       dataset-statistics definitions of Table 1 (tests/golden/)
  bruteforce_cross     pinned to scipy.sparse FP64 Q.D^T + threshold
  dense_all_pairs      a library routine (NumPy matmul) -- it is itself the pin
  graph_csr            pinned to a hand-worked graph and to scipy.sparse (A + A^T).tocsr()
  graph_knn            pinned to a hand-worked graph, tie and padding cases, and heapq
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PARTIAL_INDEX = 1
MINSIZE = 2
REMSCORE = 4
UPPERBOUND = 8
REMSCORE_FORWARD = 256  # planted mistake, tests only
ALL_PAIRS_2 = PARTIAL_INDEX | MINSIZE | REMSCORE | UPPERBOUND


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction, so every product and sum is a
    separately rounded FP64 operation)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (
        not force
        and os.path.exists(_LIB_PATH)
        and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC]
    )
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
        lib.or_result_new.restype = P
        lib.or_result_free.argtypes = [P]
        lib.or_result_count.argtypes = [P]
        lib.or_result_count.restype = i64
        lib.or_result_copy.argtypes = [P, P, P, P]
        lib.or_bruteforce.argtypes = [i32, P, P, P, f64, P]
        lib.or_bruteforce.restype = i64
        lib.or_bruteforce_rows.argtypes = [i32, P, P, P, f64, P, i32, P]
        lib.or_bruteforce_rows.restype = i64
        lib.or_bruteforce_cross.argtypes = [i32, P, P, P, i32, P, P, P, f64, P]
        lib.or_bruteforce_cross.restype = i64
        lib.or_stats.argtypes = [i32, i32, P, P, P, P, P, P, P]
        lib.or_dim_rank.argtypes = [i32, P, P]
        lib.or_rank_rows.argtypes = [i32, P, P, P, P, P, P]
        lib.or_prefix_split.argtypes = [i32, P, P, P, P, f64, P, P]
        lib.or_all_pairs.argtypes = [i32, i32, P, P, P, f64, u32, P, P, P]
        lib.or_all_pairs.restype = i64
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(c):
    ip = np.ascontiguousarray(c.indptr, dtype=np.int64)
    ix = np.ascontiguousarray(c.idx, dtype=np.int32)
    vv = np.ascontiguousarray(c.val, dtype=np.float32)
    return ip, ix, vv


class Pairs:
    """Pairs as three NumPy arrays, sorted by (i, j); scores FP64."""

    def __init__(self, i, j, s):
        o = np.lexsort((j, i))
        self.i = np.asarray(i, dtype=np.int32)[o]
        self.j = np.asarray(j, dtype=np.int32)[o]
        self.s = np.asarray(s, dtype=np.float64)[o]

    def __len__(self):
        return int(self.i.size)

    def keys(self, n: int) -> np.ndarray:
        return self.i.astype(np.int64) * int(n) + self.j.astype(np.int64)


def _collect(lib, res) -> Pairs:
    k = lib.or_result_count(res)
    i = np.empty(k, dtype=np.int32)
    j = np.empty(k, dtype=np.int32)
    s = np.empty(k, dtype=np.float64)
    if k:
        lib.or_result_copy(res, _p(i), _p(j), _p(s))
    lib.or_result_free(res)
    return Pairs(i, j, s)


def bruteforce(c, t: float) -> Pairs:
    """all-pairs-bruteforce (Sec. 4): {(i<j): dot(v_i, v_j) >= t} in FP64."""
    lib = _load()
    ip, ix, vv = _csr(c)
    res = lib.or_result_new()
    if lib.or_bruteforce(c.n, _p(ip), _p(ix), _p(vv), float(t), res) < 0:
        lib.or_result_free(res)
        raise MemoryError("oracle")
    return _collect(lib, res)


def bruteforce_rows(c, t: float, rows) -> Pairs:
    """For each listed row r: all pairs {r, j}, j != r, with dot >= t (FP64), as (min, max)."""
    lib = _load()
    ip, ix, vv = _csr(c)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    res = lib.or_result_new()
    if lib.or_bruteforce_rows(c.n, _p(ip), _p(ix), _p(vv), float(t), _p(rows), rows.size, res) < 0:
        lib.or_result_free(res)
        raise MemoryError("oracle")
    return _collect(lib, res)


def bruteforce_cross(q, c, t: float) -> Pairs:
    """Every (query row, vector id) with dot >= t (FP64)."""
    lib = _load()
    qp, qi, qv = _csr(q)
    ip, ix, vv = _csr(c)
    res = lib.or_result_new()
    r = lib.or_bruteforce_cross(q.n, _p(qp), _p(qi), _p(qv), c.n, _p(ip), _p(ix), _p(vv), float(t), res)
    if r < 0:
        lib.or_result_free(res)
        raise MemoryError("oracle")
    return _collect(lib, res)


def all_pairs(c, t: float, flags: int = ALL_PAIRS_2, query_mask=None):
    """Sequential All-Pairs (Alg. 1-2) with the paper's toggles. Returns (Pairs, counters)
    where counters = dict(visits, candidates, dots, matches, evaluations)."""
    lib = _load()
    ip, ix, vv = _csr(c)
    res = lib.or_result_new()
    cnt = np.zeros(8, dtype=np.int64)
    mask = None
    if query_mask is not None:
        mask = np.ascontiguousarray(query_mask, dtype=np.uint8)
    r = lib.or_all_pairs(
        c.n, c.m, _p(ip), _p(ix), _p(vv), float(t), int(flags),
        _p(mask) if mask is not None else None, res, _p(cnt),
    )
    if r < 0:
        lib.or_result_free(res)
        raise MemoryError("oracle")
    names = ["visits", "candidates", "dots", "matches", "evaluations"]
    return _collect(lib, res), {k: int(cnt[a]) for a, k in enumerate(names)}


def stats(c):
    """(|x|, maxweight(x), nnz per dimension, maxweight_i(V))."""
    lib = _load()
    ip, ix, vv = _csr(c)
    ln = np.empty(c.n, dtype=np.int32)
    mw = np.empty(c.n, dtype=np.float32)
    nd = np.empty(c.m, dtype=np.int32)
    md = np.empty(c.m, dtype=np.float32)
    lib.or_stats(c.n, c.m, _p(ip), _p(ix), _p(vv), _p(ln), _p(mw), _p(nd), _p(md))
    return ln, mw, nd, md


def dim_rank(nnz_d) -> np.ndarray:
    """rank[d]: position of dimension d by decreasing non-zero count, ties by id."""
    lib = _load()
    nd = np.ascontiguousarray(nnz_d, dtype=np.int32)
    rank = np.empty(nd.size, dtype=np.int32)
    lib.or_dim_rank(nd.size, _p(nd), _p(rank))
    return rank


def rank_rows(c, rank):
    """Each row's components re-expressed over ranks and sorted by rank."""
    lib = _load()
    ip, ix, vv = _csr(c)
    rk = np.ascontiguousarray(rank, dtype=np.int32)
    cr = np.empty(ix.size, dtype=np.int32)
    cv = np.empty(ix.size, dtype=np.float32)
    lib.or_rank_rows(c.n, _p(ip), _p(ix), _p(vv), _p(rk), _p(cr), _p(cv))
    return cr, cv


def prefix_split(c, t: float):
    """Partial indexing split of every row: (split = |x'|, maxweight(x')), plus the
    intermediate (rank, crank, cval, mw by rank) it was computed from."""
    lib = _load()
    ln, mw, nd, md = stats(c)
    rank = dim_rank(nd)
    mwr = np.empty(c.m, dtype=np.float32)
    mwr[rank] = md
    cr, cv = rank_rows(c, rank)
    ip = np.ascontiguousarray(c.indptr, dtype=np.int64)
    split = np.empty(c.n, dtype=np.int32)
    mwp = np.empty(c.n, dtype=np.float32)
    lib.or_prefix_split(c.n, _p(ip), _p(cr), _p(cv), _p(mwr), float(t), _p(split), _p(mwp))
    return split, mwp, {"rank": rank, "crank": cr, "cval": cv, "mwr": mwr}


def dense_all_pairs(X: np.ndarray, t: float, block: int = 4096) -> Pairs:
    """Dense form of the matrix view S = D.D^T (Sec. 2.1): FP64 matmul of the FP32
    vectors, upper triangle, S_ij >= t."""
    X64 = np.asarray(X, dtype=np.float64)
    n = X64.shape[0]
    I, J, S = [], [], []
    for a in range(0, n, block):
        blk = X64[a : a + block] @ X64.T
        r, cidx = np.nonzero(blk >= t)
        r = r + a
        keep = cidx > r
        I.append(r[keep])
        J.append(cidx[keep])
        S.append(blk[r[keep] - a, cidx[keep]])
    if not I:
        return Pairs(np.zeros(0), np.zeros(0), np.zeros(0))
    return Pairs(np.concatenate(I), np.concatenate(J), np.concatenate(S))


def dense_rows(X: np.ndarray, t: float, rows) -> Pairs:
    """Dense oracle restricted to listed rows: all {r, j}, j != r, with S_rj >= t."""
    X64 = np.asarray(X, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    blk = X64[rows] @ X64.T
    r, cidx = np.nonzero(blk >= t)
    keep = cidx != rows[r]
    a, b = rows[r[keep]], cidx[keep]
    s = blk[r[keep], cidx[keep]]
    return Pairs(np.minimum(a, b), np.maximum(a, b), s)


def graph_csr(i, j, s, n: int):
    """The similarity graph G_S(V, t) = (V, M) of Sec. 2.1: an undirected edge u <-> v of
    weight w(u, v) = u.v for every match. Rows of its adjacency, neighbours in increasing
    id: (row_ptr[n + 1], col, w)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    s = np.asarray(s, dtype=np.float32)
    src = np.concatenate([i, j])
    dst = np.concatenate([j, i])
    wt = np.concatenate([s, s])
    order = np.lexsort((dst, src))  # by vertex, then by neighbour id
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return row_ptr, dst[order].astype(np.int32), wt[order]


def graph_knn(row_ptr, col, w, k: int):
    """k-nn read off the similarity graph (Sec. 2.2): for each vertex its k neighbours of
    largest weight, ties by smaller id, padded with (-1, 0). Returns (nbr[n, k], w[n, k])."""
    n = len(row_ptr) - 1
    nbr = np.full((n, k), -1, dtype=np.int32)
    wk = np.zeros((n, k), dtype=np.float32)
    for v in range(n):
        a, b = int(row_ptr[v]), int(row_ptr[v + 1])
        c, x = col[a:b], np.asarray(w[a:b], dtype=np.float64)
        o = np.lexsort((c, -x))[:k]
        nbr[v, : len(o)] = c[o]
        wk[v, : len(o)] = x[o]
    return nbr, wk

