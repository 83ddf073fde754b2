"""The 2-D driver (Sec. 6, Alg. 7) with the GPU matcher: a 2 x 2 mesh of host ranks, each a
process using the library's join, query and exact-completion calls on the one GPU (no kernel
waits on another rank), merged on rank 0 and compared with the oracle's whole-set brute
force; once more with a rank that fails before its local pairs (recomputed by its row's
completer)."""
import multiprocessing as mp

import numpy as np
import pytest

import oracle
import synth
from parity import compare
from test_gpu_horizontal import free_port

pytestmark = pytest.mark.gpu


def gpu_worker(rank, p, q, port, t, fail, out_q):
    from datetime import timedelta

    import torch
    import torch.distributed as dist

    from paper_1402_3010_gb300 import twod as T

    torch.cuda.set_device(0)
    c, _ = synth.config_small(seed=6, n=4000, m=5000)
    store = dist.TCPStore("127.0.0.1", port, p, rank == 0, timedelta(seconds=300))
    try:
        res = T.twod_all_pairs(rank, p, q, store, c.indptr, c.idx, c.val, c.m, t, T.GpuMatcher2D(), timeout_s=15.0,
                               fail=fail)
    except RuntimeError as e:
        out_q.put((rank, "error", str(e)))
        return
    if res is not None:
        out_q.put((rank, "ok", res))


@pytest.mark.parametrize("fail", [None, (3, "before_local")])
def test_twod_gpu_2x2(fail):
    from paper_1402_3010_gb300 import _build

    _build.build()
    t = float(np.float32(0.6))
    p, q = 4, 2
    ctx = mp.get_context("spawn")
    mq = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=gpu_worker, args=(r, p, q, port, t, fail, mq)) for r in range(p)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(600)
    msgs = []
    while not mq.empty():
        msgs.append(mq.get())
    for pr in procs:
        if pr.is_alive():
            pr.kill()
    ok = [m for m in msgs if m[1] == "ok"]
    assert len(ok) == 1, msgs
    i, j, s, failed = ok[0][2]
    assert failed == ([] if fail is None else [3])
    c, _ = synth.config_small(seed=6, n=4000, m=5000)
    ref = oracle.bruteforce(c, t)
    assert len(ref.i) > 0
    compare(i, j, s, ref, t, c.n, csr=c)
