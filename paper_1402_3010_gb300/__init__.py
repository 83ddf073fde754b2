"""Python binding of libaps.so, the GB300 All-Pairs similarity join (C ABI in include/aps.h).

Argument marshalling only: every step of the join runs in the library's CUDA kernels.
Functions keep the C names. Host inputs are NumPy arrays; device inputs are PyTorch CUDA
tensors (PyTorch is used for device memory and streams only). If the compiled library
is missing this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "APSError", "load", "lib_path",
    "aps_build_index", "aps_all_pairs", "aps_query", "aps_index_export", "aps_index_info",
    "aps_index_stats", "aps_index_free", "aps_pairs_free", "aps_pairs_copy_to",
    "aps_batch_all_pairs", "aps_batch_all_pairs_csr", "aps_tune_bucket", "aps_tuning_default", "aps_get_tuning",
    "aps_set_tuning", "aps_autotune_batch_csr", "aps_all_pairs_dense", "aps_dense_tensor_products",
    "aps_server_create", "aps_stream_submit",
    "aps_stream_poll", "aps_stream_cancel", "aps_server_free", "aps_last_error", "aps_version",
    "aps_debug_fail_alloc", "aps_debug_dense_stall", "aps_debug_stage_cap", "aps_launch_count",
    "aps_all_pairs_noalloc", "pairs_to_numpy", "pairs_to_torch",
    "DEVICE_PTRS", "NORMALIZE", "QUERYABLE", "NO_PARTIAL_INDEX", "NO_MINSIZE", "NO_REMSCORE",
    "NO_UPPERBOUND", "HOST_OUTPUT",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libaps.so")

OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, EAGAIN, ETIMEOUT, ECANCELED, EUNSUPPORTED = range(9)
STATUS_NAMES = ["APS_OK", "APS_EINVAL", "APS_ENOMEM", "APS_ECUDA", "APS_EOVERFLOW", "APS_EAGAIN",
                "APS_ETIMEOUT", "APS_ECANCELED", "APS_EUNSUPPORTED"]

DEVICE_PTRS = 0x1
NORMALIZE = 0x2
QUERYABLE = 0x4
NO_PARTIAL_INDEX = 0x8
NO_MINSIZE = 0x10
NO_REMSCORE = 0x20
NO_UPPERBOUND = 0x40
HOST_OUTPUT = 0x100
SUBUNIT_NORMS = 0x200

# The paper's sequential variants (Sec. 4, Tables 2-3) as aps_build_index flag sets; the
# same values as the APS_VARIANT_* macros of aps.h.
VARIANTS = {
    "all-pairs-0-array": NO_PARTIAL_INDEX | NO_MINSIZE | NO_REMSCORE | NO_UPPERBOUND,
    "all-pairs-0-remscore": NO_PARTIAL_INDEX | NO_MINSIZE | NO_UPPERBOUND,
    "all-pairs-0-minsize": NO_PARTIAL_INDEX | NO_REMSCORE | NO_UPPERBOUND,
    "all-pairs-1-array": NO_MINSIZE | NO_REMSCORE | NO_UPPERBOUND,
    "all-pairs-1-remscore": NO_MINSIZE | NO_UPPERBOUND,
    "all-pairs-1-upperbound": NO_MINSIZE | NO_REMSCORE,
    "all-pairs-1-minsize": NO_REMSCORE | NO_UPPERBOUND,
    "all-pairs-1-remscore-minsize": NO_UPPERBOUND,
    "all-pairs-2": 0,
}

_P = ctypes.c_void_p
_i32, _i64, _u32, _u64, _f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float


class aps_pairs(ctypes.Structure):
    _fields_ = [("count", _i64), ("i", _P), ("j", _P), ("score", _P), ("on_device", _i32),
                ("_reserved", _i32), ("_priv", _P)]


class aps_graph(ctypes.Structure):
    _fields_ = [("n", _i32), ("on_device", _i32), ("nnz", _i64), ("row_ptr", _P), ("col", _P), ("w", _P),
                ("_priv", _P)]


TUNE_BUCKETS = 8
TUNE_BOUNDS = (512, 1280, 2560, 5120, 10240, 20480, 40960, None)  # None: unbounded


class aps_tuning(ctypes.Structure):
    _fields_ = [("groups", _i32 * TUNE_BUCKETS), ("query_groups", _i32 * TUNE_BUCKETS)]


class aps_tune_report(ctypes.Structure):
    _fields_ = [("instances", _i32 * TUNE_BUCKETS), ("sampled", _i32 * TUNE_BUCKETS),
                ("ms", (_f32 * 4) * TUNE_BUCKETS), ("ms_default", _f32), ("ms_tuned", _f32),
                ("kept_default", _i32), ("_reserved", _i32)]

    def as_dict(self):
        return {"instances": list(self.instances), "sampled": list(self.sampled),
                "ms": [[round(float(v), 4) for v in row] for row in self.ms],
                "ms_default": float(self.ms_default), "ms_tuned": float(self.ms_tuned),
                "kept_default": int(self.kept_default)}


class aps_stats(ctypes.Structure):
    _fields_ = [("visits", _i64), ("candidates", _i64), ("verified", _i64), ("pairs", _i64),
                ("band", _i64), ("evaluations", _i64), ("reruns", _i64), ("ms_build", _f32),
                ("ms_join", _f32), ("ms_sort", _f32), ("ms_total", _f32), ("entries_read", _i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class aps_timeline(ctypes.Structure):
    _fields_ = [("batches", _i64), ("busy_ms", ctypes.c_double), ("overlap_ms", ctypes.c_double),
                ("span_ms", ctypes.c_double), ("max_in_flight", _i32), ("_reserved", _i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("_")}


class aps_instance(ctypes.Structure):
    _fields_ = [("indptr", _P), ("idx", _P), ("val", _P), ("n", _i32), ("m", _i32), ("t", _f32),
                ("_reserved", _i32)]


class aps_query_req(ctypes.Structure):
    _fields_ = [("qptr", _P), ("qidx", _P), ("qval", _P), ("nq", _i32), ("t", _f32)]


class APSError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {aps_last_error()}")


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libaps.so (built by __graft_entry__.build() or paper_1402_3010_gb300._build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(_LIB_PATH)
        sigs = {
            "aps_build_index": (_i32, [_P, _P, _P, _i32, _i32, _f32, _u32, _P, ctypes.POINTER(_P)]),
            "aps_all_pairs": (_i32, [_P, _u32, ctypes.POINTER(aps_pairs)]),
            "aps_all_pairs_split": (_i32, [_P, _i32, _i64, _u32, ctypes.POINTER(aps_pairs)]),
            "aps_query": (_i32, [_P, _P, _P, _P, _i32, _f32, _u32, ctypes.POINTER(aps_pairs)]),
            "aps_index_export": (_i32, [_P] + [_P] * 13),
            "aps_index_info": (_i32, [_P, _P, _P, _P, _P]),
            "aps_index_stats": (_i32, [_P, ctypes.POINTER(aps_stats)]),
            "aps_index_free": (None, [_P]),
            "aps_pairs_free": (None, [ctypes.POINTER(aps_pairs)]),
            "aps_pairs_copy_to": (_i32, [ctypes.POINTER(aps_pairs), _P, _P, _P, _P]),
            "aps_batch_all_pairs": (_i32, [_i32, ctypes.POINTER(aps_instance), _u32, _P,
                                           ctypes.POINTER(aps_pairs), ctypes.POINTER(aps_stats)]),
            "aps_tune_bucket": (_i32, [_i64]),
            "aps_tuning_default": (None, [ctypes.POINTER(aps_tuning)]),
            "aps_get_tuning": (None, [ctypes.POINTER(aps_tuning)]),
            "aps_set_tuning": (_i32, [ctypes.POINTER(aps_tuning)]),
            "aps_autotune_batch_csr": (_i32, [_i32, _P, _P, _P, _P, _P, _P, _u32, _P, ctypes.POINTER(aps_tuning),
                                              ctypes.POINTER(aps_tune_report)]),
            "aps_batch_all_pairs_csr": (_i32, [_i32, _P, _P, _P, _P, _P, _P, _u32, _P, ctypes.POINTER(aps_pairs),
                                               ctypes.POINTER(aps_stats)]),
            "aps_dense_tensor_products": (_i32, [_P, _i32, _i32, _P, _P]),
            "aps_all_pairs_dense": (_i32, [_P, _i32, _i32, _f32, _u32, _P, ctypes.POINTER(aps_pairs),
                                           ctypes.POINTER(aps_stats)]),
            "aps_server_create": (_i32, [_P, ctypes.c_size_t, _i32, ctypes.POINTER(_P)]),
            "aps_stream_submit": (_i32, [_P, ctypes.POINTER(aps_query_req), ctypes.POINTER(_u64)]),
            "aps_stream_poll": (_i32, [_P, _u64, _i32, ctypes.POINTER(aps_pairs)]),
            "aps_stream_cancel": (_i32, [_P, _u64]),
            "aps_server_free": (None, [_P]),
            "aps_server_timeline": (_i32, [_P, ctypes.POINTER(aps_timeline)]),
            "aps_last_error": (ctypes.c_char_p, []),
            "aps_version": (ctypes.c_char_p, []),
            "aps_debug_fail_alloc": (None, [_i64]),
            "aps_debug_dense_stall": (None, [_i64, _u64]),
            "aps_debug_stage_cap": (None, [_i64]),
            "aps_launch_count": (_i64, []),
            "aps_all_pairs_noalloc": (_i32, [_P, _P, _P, _P, _i64, ctypes.POINTER(_i64), _P]),
            "aps_graph_csr": (_i32, [_P, _P, _P, _i64, _i32, _u32, _P, ctypes.POINTER(aps_graph)]),
            "aps_graph_knn": (_i32, [ctypes.POINTER(aps_graph), _i32, _P, _P, _u32, _P]),
            "aps_graph_copy_to": (_i32, [ctypes.POINTER(aps_graph), _P, _P, _P, _P]),
            "aps_graph_free": (None, [ctypes.POINTER(aps_graph)]),
            "aps_pairs_verify": (_i32, [ctypes.POINTER(aps_pairs), _i32, _P, _P, _P, _i32, _i32, _f32, _u32, _P,
                                        ctypes.POINTER(aps_pairs), ctypes.POINTER(_i64)]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def aps_last_error() -> str:
    if _lib is None:
        return ""
    v = _lib.aps_last_error()
    return v.decode() if v else ""


def aps_version() -> str:
    return load().aps_version().decode()


def aps_launch_count() -> int:
    return int(load().aps_launch_count())


def aps_debug_fail_alloc(k: int) -> None:
    load().aps_debug_fail_alloc(int(k))


def aps_debug_dense_stall(launches: int, wait_ns: int = 0) -> None:
    load().aps_debug_dense_stall(int(launches), int(wait_ns))


def aps_debug_stage_cap(pairs: int) -> None:
    load().aps_debug_stage_cap(int(pairs))


def _check(st: int, where: str):
    if st != OK:
        raise APSError(st, where)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _csr_args(indptr, idx, val):
    """(pointers, flags, keep-alive) for host NumPy or device torch CSR arrays."""
    if _is_torch(indptr):
        for a, dt in ((indptr, "int64"), (idx, "int32"), (val, "float32")):
            if not a.is_cuda or str(a.dtype) != f"torch.{dt}" or not a.is_contiguous():
                raise TypeError(f"device CSR arrays must be contiguous CUDA {dt} tensors")
        return (_ptr(indptr), _ptr(idx), _ptr(val)), DEVICE_PTRS, (indptr, idx, val)
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(idx, dtype=np.int32)
    vv = np.ascontiguousarray(val, dtype=np.float32)
    return (ip.ctypes.data, ix.ctypes.data, vv.ctypes.data), 0, (ip, ix, vv)


def aps_build_index(indptr, idx, val, n: int, m: int, t: float, flags: int = 0, stream=None) -> int:
    """Build the index; returns an opaque handle (int). Free with aps_index_free."""
    lib = load()
    (p0, p1, p2), f, keep = _csr_args(indptr, idx, val)
    out = _P()
    st = lib.aps_build_index(p0, p1, p2, int(n), int(m), float(t), int(flags) | f, _stream_ptr(stream),
                             ctypes.byref(out))
    del keep
    _check(st, "aps_build_index")
    return out.value


def aps_all_pairs(index: int, flags: int = 0) -> aps_pairs:
    lib = load()
    out = aps_pairs()
    _check(lib.aps_all_pairs(index, int(flags), ctypes.byref(out)), "aps_all_pairs")
    return out


def aps_all_pairs_split(index: int, nblk: int, heavy: int, flags: int = 0) -> aps_pairs:
    """The self-join with the `heavy` costliest vectors joined as nblk dimension blocks
    each (the vertical algorithm's local pruning inside the join); same pairs as
    aps_all_pairs."""
    lib = load()
    out = aps_pairs()
    _check(lib.aps_all_pairs_split(index, int(nblk), int(heavy), int(flags), ctypes.byref(out)),
           "aps_all_pairs_split")
    return out


def aps_query(index: int, qptr, qidx, qval, nq: int, t: float, flags: int = 0) -> aps_pairs:
    lib = load()
    (p0, p1, p2), f, keep = _csr_args(qptr, qidx, qval)
    out = aps_pairs()
    st = lib.aps_query(index, p0, p1, p2, int(nq), float(t), int(flags) | f, ctypes.byref(out))
    del keep
    _check(st, "aps_query")
    return out


def aps_all_pairs_noalloc(index: int, i, j, score, stream=None) -> int:
    """Self-join into caller-owned CUDA int32/int32/float32 tensors of equal length (the
    capacity), with no allocation inside the library; returns the number of pairs.
    APSError with status EOVERFLOW carries the needed count in .count."""
    # The kernels write these arrays from the device: anything but contiguous CUDA tensors
    # of the right type (a NumPy array, a CPU tensor, int16 or a strided view) would make
    # them write to host memory or past the caller's storage.
    for a, dt, nm in ((i, "int32", "i"), (j, "int32", "j"), (score, "float32", "score")):
        if not _is_torch(a) or not a.is_cuda:
            raise ValueError(f"{nm} must be a CUDA tensor (got {type(a).__name__})")
        if str(a.dtype) != f"torch.{dt}" or not a.is_contiguous():
            raise ValueError(f"{nm} must be a contiguous {dt} CUDA tensor (got {a.dtype}, "
                             f"contiguous={a.is_contiguous()})")
    if not (i.device == j.device == score.device):
        raise ValueError("i, j and score must be on the same CUDA device")
    cap = int(i.numel())
    if int(j.numel()) != cap or int(score.numel()) != cap:
        raise ValueError("i, j and score must have the same length")
    cnt = _i64(0)
    st = load().aps_all_pairs_noalloc(index, _ptr(i) if cap else None, _ptr(j) if cap else None,
                                      _ptr(score) if cap else None, cap, ctypes.byref(cnt), _stream_ptr(stream))
    if st != OK:
        err = APSError(st, "aps_all_pairs_noalloc")
        err.count = cnt.value
        raise err
    return cnt.value


def aps_index_info(index: int) -> dict:
    lib = load()
    n, m, nnz, ind = _i32(), _i32(), _i64(), _i64()
    _check(lib.aps_index_info(index, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nnz), ctypes.byref(ind)),
           "aps_index_info")
    return {"n": n.value, "m": m.value, "nnz": nnz.value, "indexed": ind.value}


def aps_index_export(index: int) -> dict:
    info = aps_index_info(index)
    n, m, nnz, nsuf = info["n"], info["m"], info["nnz"], info["indexed"]
    out = {
        "len": np.empty(n, np.int32), "mw": np.empty(n, np.float32), "nnz_d": np.empty(m, np.int32),
        "mw_d": np.empty(m, np.float32), "rank_of_dim": np.empty(m, np.int32),
        "crank": np.empty(nnz, np.int32), "cval": np.empty(nnz, np.float32), "split": np.empty(n, np.int32),
        "qsplit": np.empty(n, np.int32), "mw_pre": np.empty(n, np.float32), "list_ptr": np.empty(m + 1, np.int64),
        "post_id": np.empty(nsuf, np.int32), "post_w": np.empty(nsuf, np.float32),
    }
    order = ["len", "mw", "nnz_d", "mw_d", "rank_of_dim", "crank", "cval", "split", "qsplit", "mw_pre",
             "list_ptr", "post_id", "post_w"]
    _check(load().aps_index_export(index, *[out[k].ctypes.data for k in order]), "aps_index_export")
    return out


def aps_index_stats(index: int) -> dict:
    s = aps_stats()
    _check(load().aps_index_stats(index, ctypes.byref(s)), "aps_index_stats")
    return s.as_dict()


def aps_index_free(index: int) -> None:
    if index:
        load().aps_index_free(index)


def aps_pairs_free(p: aps_pairs) -> None:
    load().aps_pairs_free(ctypes.byref(p))


def aps_pairs_copy_to(p: aps_pairs, i, j, score, stream=None) -> None:
    _check(load().aps_pairs_copy_to(ctypes.byref(p), _ptr(i), _ptr(j), _ptr(score), _stream_ptr(stream)),
           "aps_pairs_copy_to")


def pairs_to_numpy(p: aps_pairs):
    """(i, j, score) NumPy copies of a result."""
    n = int(p.count)
    i = np.empty(n, np.int32)
    j = np.empty(n, np.int32)
    s = np.empty(n, np.float32)
    if n:
        aps_pairs_copy_to(p, i, j, s)
    return i, j, s


def pairs_to_torch(p: aps_pairs, device="cuda"):
    """(i, j, score) torch CUDA tensors copied from a result."""
    import torch

    n = int(p.count)
    i = torch.empty(n, dtype=torch.int32, device=device)
    j = torch.empty(n, dtype=torch.int32, device=device)
    s = torch.empty(n, dtype=torch.float32, device=device)
    if n:
        aps_pairs_copy_to(p, i, j, s, torch.cuda.current_stream(device))
    return i, j, s


def aps_batch_all_pairs(instances, flags: int = 0, stream=None):
    """instances: list of (indptr, idx, val, n, m, t) (NumPy host or torch device arrays).
    Returns (list of aps_pairs, stats dict)."""
    lib = load()
    k = len(instances)
    arr = (aps_instance * k)()
    keep = []
    f = 0
    for a, (ip, ix, vv, n, m, t) in enumerate(instances):
        (p0, p1, p2), f, kp = _csr_args(ip, ix, vv)
        keep.append(kp)
        arr[a].indptr, arr[a].idx, arr[a].val = p0, p1, p2
        arr[a].n, arr[a].m, arr[a].t = int(n), int(m), float(t)
    outs = (aps_pairs * k)()
    st = aps_stats()
    rc = lib.aps_batch_all_pairs(k, arr, int(flags) | f, _stream_ptr(stream), outs, ctypes.byref(st))
    del keep
    _check(rc, "aps_batch_all_pairs")
    return list(outs), st.as_dict()


def aps_batch_all_pairs_csr(row_offsets, indptr, idx, val, m, t, flags: int = 0, stream=None):
    """One concatenated CSR (NumPy host or torch device arrays) with instance row offsets
    (host int64 [k+1]), per-instance m (int32 [k]) and t (float32 [k]).
    Returns (list of aps_pairs, stats dict)."""
    lib = load()
    ro = np.ascontiguousarray(row_offsets, dtype=np.int64)
    mm = np.ascontiguousarray(m, dtype=np.int32)
    tt = np.ascontiguousarray(t, dtype=np.float32)
    k = int(ro.size - 1)
    (p0, p1, p2), f, keep = _csr_args(indptr, idx, val)
    outs = (aps_pairs * k)()
    st = aps_stats()
    rc = lib.aps_batch_all_pairs_csr(k, ro.ctypes.data, p0, p1, p2, mm.ctypes.data, tt.ctypes.data, int(flags) | f,
                                     _stream_ptr(stream), outs, ctypes.byref(st))
    del keep
    _check(rc, "aps_batch_all_pairs_csr")
    return list(outs), st.as_dict()


def aps_tune_bucket(n: int) -> int:
    return int(load().aps_tune_bucket(int(n)))


def aps_tuning_default(query: bool = False) -> list:
    """The built-in table's self-join column (query=True: its queryable-index column)."""
    tu = aps_tuning()
    load().aps_tuning_default(ctypes.byref(tu))
    return list(tu.query_groups if query else tu.groups)


def aps_get_tuning(query: bool = False) -> list:
    """The table in force: its self-join column (query=True: its queryable-index column)."""
    tu = aps_tuning()
    load().aps_get_tuning(ctypes.byref(tu))
    return list(tu.query_groups if query else tu.groups)


def aps_set_tuning(groups, query_groups=None) -> None:
    """groups: TUNE_BUCKETS query-group counts (1, 2, 4 or 8), one per size bucket, for
    self-joins; query_groups: the same for indexes built with QUERYABLE (None: unchanged)."""
    cur = aps_tuning()
    load().aps_get_tuning(ctypes.byref(cur))
    cols = {"groups": groups, "query_groups": query_groups if query_groups is not None else list(cur.query_groups)}
    tu = aps_tuning()
    for name, vals in cols.items():
        v = list(vals)
        if len(v) != TUNE_BUCKETS:
            raise ValueError(f"need {TUNE_BUCKETS} entries")
        arr = getattr(tu, name)
        for b, x in enumerate(v):
            arr[b] = int(x)
    _check(load().aps_set_tuning(ctypes.byref(tu)), "aps_set_tuning")


def aps_autotune_batch_csr(row_offsets, indptr, idx, val, m, t, flags: int = 0, stream=None):
    """Time the join of each size bucket's sample under G = 1, 2, 4, 8 and install the
    fastest table (arguments as aps_batch_all_pairs_csr). Returns (groups, report dict)."""
    lib = load()
    ro = np.ascontiguousarray(row_offsets, dtype=np.int64)
    mm = np.ascontiguousarray(m, dtype=np.int32)
    tt = np.ascontiguousarray(t, dtype=np.float32)
    k = int(ro.size - 1)
    (p0, p1, p2), f, keep = _csr_args(indptr, idx, val)
    tu = aps_tuning()
    rep = aps_tune_report()
    rc = lib.aps_autotune_batch_csr(k, ro.ctypes.data, p0, p1, p2, mm.ctypes.data, tt.ctypes.data, int(flags) | f,
                                    _stream_ptr(stream), ctypes.byref(tu), ctypes.byref(rep))
    del keep
    _check(rc, "aps_autotune_batch_csr")
    return list(tu.groups), rep.as_dict()


def aps_all_pairs_dense(X, t: float, flags: int = 0, stream=None):
    """X: float32 [n, d] NumPy (host) or torch CUDA tensor. Returns (aps_pairs, stats dict)."""
    lib = load()
    if _is_torch(X):
        if not X.is_cuda or str(X.dtype) != "torch.float32" or not X.is_contiguous():
            raise TypeError("X must be a contiguous CUDA float32 tensor")
        f = DEVICE_PTRS
        ptr = X.data_ptr()
    else:
        X = np.ascontiguousarray(X, dtype=np.float32)
        f = 0
        ptr = X.ctypes.data
    n, d = X.shape
    out = aps_pairs()
    st = aps_stats()
    _check(lib.aps_all_pairs_dense(ptr, int(n), int(d), float(t), int(flags) | f, _stream_ptr(stream),
                                   ctypes.byref(out), ctypes.byref(st)), "aps_all_pairs_dense")
    return out, st.as_dict()


def aps_dense_tensor_products(X, raw, stream=None) -> None:
    """X: contiguous CUDA float32 [n, d]; raw: contiguous CUDA float32 [n, n], receiving the
    tensor cores' float32 products of the dense path's computed blocks."""
    for a in (X, raw):
        if not _is_torch(a) or not a.is_cuda or str(a.dtype) != "torch.float32" or not a.is_contiguous():
            raise TypeError("X and raw must be contiguous CUDA float32 tensors")
    n, d = X.shape
    if tuple(raw.shape) != (n, n):
        raise ValueError("raw must be n x n")
    _check(load().aps_dense_tensor_products(X.data_ptr(), int(n), int(d), raw.data_ptr(), _stream_ptr(stream)),
           "aps_dense_tensor_products")


def aps_server_create(index: int, mem_budget: int, slots: int) -> int:
    out = _P()
    _check(load().aps_server_create(index, int(mem_budget), int(slots), ctypes.byref(out)), "aps_server_create")
    return out.value


def aps_stream_submit(server: int, qptr, qidx, qval, nq: int, t: float) -> int:
    ip = np.ascontiguousarray(qptr, dtype=np.int64)
    ix = np.ascontiguousarray(qidx, dtype=np.int32)
    vv = np.ascontiguousarray(qval, dtype=np.float32)
    req = aps_query_req(ip.ctypes.data, ix.ctypes.data, vv.ctypes.data, int(nq), float(t))
    ticket = _u64()
    _check(load().aps_stream_submit(server, ctypes.byref(req), ctypes.byref(ticket)), "aps_stream_submit")
    return ticket.value


def aps_stream_poll(server: int, ticket: int, timeout_us: int = 0):
    """Returns aps_pairs when done, None while the request is still running."""
    out = aps_pairs()
    st = load().aps_stream_poll(server, int(ticket), int(timeout_us), ctypes.byref(out))
    if st == EAGAIN:
        return None
    _check(st, "aps_stream_poll")
    return out


def aps_stream_cancel(server: int, ticket: int) -> None:
    _check(load().aps_stream_cancel(server, int(ticket)), "aps_stream_cancel")


def aps_server_timeline(server: int) -> dict:
    """The device time line of the server's completed batches: batches, busy_ms (at least
    one batch in flight), overlap_ms (two or more), span_ms, max_in_flight."""
    st = aps_timeline()
    _check(load().aps_server_timeline(server, ctypes.byref(st)), "aps_server_timeline")
    return st.as_dict()


def aps_server_free(server: int) -> None:
    if server:
        load().aps_server_free(server)


def aps_graph_csr(i, j=None, s=None, n: int = 0, flags: int = 0, stream=None) -> aps_graph:
    """CSR adjacency of the similarity graph from a pair list: an aps_pairs result, or
    i, j, s as host NumPy or device torch arrays (int32, int32, float32)."""
    lib = load()
    g = aps_graph()
    if isinstance(i, aps_pairs):
        p = i
        ptrs, count = (p.i, p.j, p.score), int(p.count)
        flags |= DEVICE_PTRS if p.on_device else 0
        keep = (p,)
    elif _is_torch(i):
        for a, dt in ((i, "int32"), (j, "int32"), (s, "float32")):
            if not a.is_cuda or str(a.dtype) != f"torch.{dt}" or not a.is_contiguous():
                raise TypeError(f"device pair arrays must be contiguous CUDA {dt} tensors")
        ptrs, count, keep = (_ptr(i), _ptr(j), _ptr(s)), int(i.numel()), (i, j, s)
        flags |= DEVICE_PTRS
    else:
        a = np.ascontiguousarray(i, dtype=np.int32)
        b = np.ascontiguousarray(j, dtype=np.int32)
        c = np.ascontiguousarray(s, dtype=np.float32)
        ptrs, count, keep = (a.ctypes.data, b.ctypes.data, c.ctypes.data), int(a.size), (a, b, c)
    _check(lib.aps_graph_csr(*ptrs, count, int(n), flags, _stream_ptr(stream), ctypes.byref(g)), "aps_graph_csr")
    del keep
    return g


def aps_graph_knn(g: aps_graph, k: int, nbr=None, wk=None, stream=None):
    """k nearest neighbours per vertex: (nbr[n, k], wk[n, k]); NumPy host arrays unless
    torch CUDA tensors are passed in."""
    lib = load()
    flags = 0
    if nbr is None:
        nbr = np.empty((g.n, k), np.int32)
        wk = np.empty((g.n, k), np.float32)
    elif _is_torch(nbr):
        flags |= DEVICE_PTRS
    _check(lib.aps_graph_knn(ctypes.byref(g), int(k), _ptr(nbr), _ptr(wk), flags, _stream_ptr(stream)),
           "aps_graph_knn")
    return nbr, wk


def graph_to_numpy(g: aps_graph):
    """(row_ptr, col, w) NumPy copies of a graph."""
    rp = np.empty(g.n + 1, np.int64)
    col = np.empty(g.nnz, np.int32)
    w = np.empty(g.nnz, np.float32)
    _check(load().aps_graph_copy_to(ctypes.byref(g), rp.ctypes.data, col.ctypes.data, w.ctypes.data, None),
           "aps_graph_copy_to")
    return rp, col, w


def aps_graph_free(g: aps_graph) -> None:
    load().aps_graph_free(ctypes.byref(g))


def aps_pairs_verify(lists, indptr, idx, val, n: int, m: int, t: float, flags: int = 0, stream=None):
    """Union of candidate pair lists (aps_pairs results), each pair rescored exactly from
    the rows (host NumPy or device torch CSR); returns (aps_pairs of dot >= t, union size)."""
    lib = load()
    arr = (aps_pairs * max(len(lists), 1))()
    for k, p in enumerate(lists):
        arr[k] = p
    (ip, ix, vv), f, keep = _csr_args(indptr, idx, val)
    out = aps_pairs()
    nc = _i64(0)
    _check(lib.aps_pairs_verify(arr, len(lists), ip, ix, vv, int(n), int(m), float(t), flags | f,
                                _stream_ptr(stream), ctypes.byref(out), ctypes.byref(nc)), "aps_pairs_verify")
    del keep
    return out, int(nc.value)

