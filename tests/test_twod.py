"""Host logic of the 2-D driver (Sec. 6, Alg. 7) on meshes of 2-4 ranks on CPU: real
processes and a real TCPStore, an oracle-backed matcher in place of the GPU, and host-side
faults (a rank that raises before publishing its projection or its local pairs, a row
completer that raises, a rank that never joins). The merged result must equal the oracle's
whole-set brute force."""
import multiprocessing as mp

import numpy as np
import pytest

import oracle
import synth
from parity import compare
from test_horizontal import free_port


class OracleMatcher2D:
    """CPU stand-in for the GPU matcher: the oracle's brute force on the projections at the
    local threshold, and float64 rescoring of the union from the full rows."""

    def local(self, part, lower, t_local):
        c = synth.SparseCSR(part.indptr, part.idx, part.val, part.n, part.m)
        r = oracle.bruteforce(c, t_local)
        own = (r.i.astype(np.int64), r.j.astype(np.int64), r.s.astype(np.float32))
        cross = []
        for q in lower:
            qc = synth.SparseCSR(q.indptr, q.idx, q.val, q.n, q.m)
            x = oracle.bruteforce_cross(qc, c, t_local)
            cross.append((x.i.astype(np.int64), x.j.astype(np.int64), x.s.astype(np.float32)))
        return own, cross

    def complete(self, ci, cj, rows, t):
        keys = np.unique(np.asarray(ci, np.int64) * rows.n + np.asarray(cj, np.int64))
        i, j = keys // rows.n, keys % rows.n
        dense = np.zeros((rows.n, rows.m))
        for k in range(rows.n):
            a, b = rows.indptr[k], rows.indptr[k + 1]
            dense[k, rows.idx[a:b]] = rows.val[a:b]
        s = np.einsum("ij,ij->i", dense[i], dense[j]) if keys.size else np.zeros(0)
        keep = s >= t
        return i[keep], j[keep], s[keep].astype(np.float32)


def worker(rank, p, q, port, t, fail, skip, out_q, seed):
    from datetime import timedelta

    import torch.distributed as dist

    from paper_1402_3010_gb300 import twod as T

    c, _ = synth.config_small(seed=seed, n=600, m=1200)
    store = dist.TCPStore("127.0.0.1", port, p, rank == 0, timedelta(seconds=60))
    if skip == rank:  # this rank never takes part
        return
    try:
        res = T.twod_all_pairs(rank, p, q, store, c.indptr, c.idx, c.val, c.m, t, OracleMatcher2D(),
                               timeout_s=3.0, fail=fail)
    except RuntimeError as e:
        out_q.put((rank, "error", str(e)))
        return
    if res is not None:
        out_q.put((rank, "ok", res))


def run(p, q, fail=None, skip=None, seed=3, t=0.6):
    ctx = mp.get_context("spawn")
    mq = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, p, q, port, t, fail, skip, mq, seed)) for r in range(p)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(180)
    msgs = []
    while not mq.empty():
        msgs.append(mq.get())
    for pr in procs:
        if pr.is_alive():
            pr.kill()
    return msgs


def check(msgs, t, seed=3, failed=()):
    ok = [m for m in msgs if m[1] == "ok"]
    assert len(ok) == 1 and ok[0][0] == 0
    i, j, s, got_failed = ok[0][2]
    assert sorted(got_failed) == sorted(failed)
    c, _ = synth.config_small(seed=seed, n=600, m=1200)
    ref = oracle.bruteforce(c, t)
    assert len(ref.i) > 0
    compare(i, j, s, ref, t, c.n, csr=c)


@pytest.mark.parametrize("p,q", [(1, 1), (2, 2), (2, 1), (4, 2)])
def test_twod_matches_whole_set(p, q):
    t = float(np.float32(0.6))
    check(run(p, q, t=t), t)


def test_rank_failing_before_its_local_pairs_is_recomputed():
    t = float(np.float32(0.6))
    msgs = run(4, 2, fail=(3, "before_local"), t=t)
    assert any(m[0] == 3 and m[1] == "error" for m in msgs)
    check(msgs, t, failed=[3])


def test_rank_failing_before_publishing_its_projection():
    t = float(np.float32(0.6))
    check(run(4, 2, fail=(1, "before_part"), t=t), t, failed=[1])


def test_row_completer_failing_is_recomputed_by_the_collector():
    t = float(np.float32(0.6))
    msgs = run(4, 2, fail=(2, "before_row"), t=t)
    check(msgs, t, failed=[2])


def test_rank_that_never_joins():
    t = float(np.float32(0.6))
    check(run(4, 2, skip=3, t=t), t, failed=[3])


def test_mesh_parts_cover_the_set():
    from paper_1402_3010_gb300 import twod as T
    from paper_1402_3010_gb300.horizontal import cyclic_part

    c, _ = synth.config_small(seed=4, n=101, m=300)
    block = T.dimension_blocks(c.indptr, c.idx, c.m, 3)
    tot = 0
    for a in range(2):
        rows = cyclic_part(c.indptr, c.idx, c.val, c.m, a, 2)
        parts = [T.block_part(rows, block, k) for k in range(3)]
        assert sum(int(x.idx.size) for x in parts) == rows.idx.size
        for k, x in enumerate(parts):
            assert np.all(block[x.idx] == k)
        tot += rows.idx.size
    assert tot == c.idx.size
    with pytest.raises(ValueError):
        T.mesh_shape(6, 4)
