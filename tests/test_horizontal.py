"""Host logic of the horizontal driver (Sec. 5.2, Alg. 6) with world size 2-3 on CPU:
real processes and a real TCPStore, an oracle-backed matcher in place of the GPU, and
host-side faults (a rank that raises before or after publishing its vectors, a rank that
never joins). The merged result must equal the oracle's whole-set brute force."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from parity import compare


class OracleMatcher:
    """CPU stand-in for the GPU matcher: the oracle's brute force on the same parts."""

    def self_and_cross(self, part, lower, t):
        c = synth.SparseCSR(part.indptr, part.idx, part.val, part.n, part.m)
        r = oracle.bruteforce(c, t)
        own = (r.i.astype(np.int64), r.j.astype(np.int64), r.s.astype(np.float32))
        cross = []
        for q in lower:
            qc = synth.SparseCSR(q.indptr, q.idx, q.val, q.n, q.m)
            x = oracle.bruteforce_cross(qc, c, t)
            cross.append((x.i.astype(np.int64), x.j.astype(np.int64), x.s.astype(np.float32)))
        return own, cross


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, p, port, t, fail, skip, out_q, seed):
    from datetime import timedelta

    import torch.distributed as dist

    from paper_1402_3010_gb300 import horizontal as H

    c, _ = synth.config_small(seed=seed, n=900, m=1500)
    store = dist.TCPStore("127.0.0.1", port, p, rank == 0, timedelta(seconds=60))
    if skip == rank:  # this rank never takes part
        return
    part_of = lambda r: H.cyclic_part(c.indptr, c.idx, c.val, c.m, r, p)  # noqa: E731
    try:
        res = H.horizontal_all_pairs(rank, p, store, part_of, t, OracleMatcher(), timeout_s=3.0, fail=fail)
    except RuntimeError as e:
        out_q.put((rank, "error", str(e)))
        return
    if res is not None:
        out_q.put((rank, "ok", res))


def run(p, fail=None, skip=None, seed=3, t=0.6):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, p, port, t, fail, skip, q, seed)) for r in range(p)]
    for pr in procs:
        pr.start()
    msgs = []
    for pr in procs:
        pr.join(120)
    while not q.empty():
        msgs.append(q.get())
    for pr in procs:
        if pr.is_alive():
            pr.kill()
    return msgs


def check(msgs, t, seed=3, failed=()):
    ok = [m for m in msgs if m[1] == "ok"]
    assert len(ok) == 1 and ok[0][0] == 0
    i, j, s, got_failed = ok[0][2]
    assert sorted(got_failed) == sorted(failed)
    c, _ = synth.config_small(seed=seed, n=900, m=1500)
    ref = oracle.bruteforce(c, t)
    assert len(ref.i) > 0
    compare(i, j, s, ref, t, c.n, csr=c)


@pytest.mark.parametrize("p", [2, 3])
def test_horizontal_matches_whole_set(p):
    t = float(np.float32(0.6))
    check(run(p, t=t), t)


def test_rank_failing_after_publishing_is_recomputed():
    t = float(np.float32(0.6))
    msgs = run(2, fail=(1, "before_result"), t=t)
    assert any(m[0] == 1 and m[1] == "error" for m in msgs)
    check(msgs, t, failed=[1])


def test_rank_failing_before_publishing_is_recomputed():
    t = float(np.float32(0.6))
    msgs = run(3, fail=(1, "before_part"), t=t)
    check(msgs, t, failed=[1])


def test_rank_that_never_joins():
    t = float(np.float32(0.6))
    check(run(3, skip=2, t=t), t, failed=[2])


def test_cyclic_parts_cover_the_set():
    from paper_1402_3010_gb300 import horizontal as H

    c, _ = synth.config_small(seed=4, n=101, m=300)
    parts = [H.cyclic_part(c.indptr, c.idx, c.val, c.m, r, 4) for r in range(4)]
    g = np.sort(np.concatenate([q.gids for q in parts]))
    assert np.array_equal(g, np.arange(101))
    for q in parts:
        for k, gid in enumerate(q.gids):
            a, b = c.indptr[gid], c.indptr[gid + 1]
            assert np.array_equal(q.idx[q.indptr[k]:q.indptr[k + 1]], c.idx[a:b])


def test_store_values_larger_than_a_piece_round_trip():
    from datetime import timedelta

    import torch.distributed as dist

    from paper_1402_3010_gb300 import horizontal as H

    store = dist.TCPStore("127.0.0.1", free_port(), 1, True, timedelta(seconds=30))
    big = np.random.default_rng(0).integers(0, 1 << 30, size=11_000_000, dtype=np.int64)  # 88 MB
    H._put(store, "k", big)
    got = H._get(store, "k", 5.0)
    assert np.array_equal(got, big)
    assert H._get(store, "missing", 0.5) is None
