"""The horizontal driver (Sec. 5.2, Alg. 6) with the GPU matcher: two host ranks, each a
process using the library's join and query path on the one GPU (no kernel waits on the
other rank), merged on rank 0 and compared with the oracle's whole-set brute force."""
import multiprocessing as mp
import socket

import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def gpu_worker(rank, p, port, t, fail, out_q):
    from datetime import timedelta

    import torch
    import torch.distributed as dist

    from paper_1402_3010_gb300 import horizontal as H

    torch.cuda.set_device(0)
    c, _ = synth.config_small(seed=6, n=4000, m=5000)
    store = dist.TCPStore("127.0.0.1", port, p, rank == 0, timedelta(seconds=120))
    part_of = lambda r: H.cyclic_part(c.indptr, c.idx, c.val, c.m, r, p)  # noqa: E731
    try:
        res = H.horizontal_all_pairs(rank, p, store, part_of, t, H.GpuMatcher(), timeout_s=20.0, fail=fail)
    except RuntimeError as e:
        out_q.put((rank, "error", str(e)))
        return
    if res is not None:
        out_q.put((rank, "ok", res))


@pytest.mark.parametrize("fail", [None, (1, "before_result")])
def test_horizontal_gpu_two_ranks(fail):
    from paper_1402_3010_gb300 import _build

    _build.build()
    t = float(np.float32(0.6))
    p = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=gpu_worker, args=(r, p, port, t, fail, q)) for r in range(p)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(300)
    msgs = []
    while not q.empty():
        msgs.append(q.get())
    for pr in procs:
        if pr.is_alive():
            pr.kill()
    ok = [m for m in msgs if m[1] == "ok"]
    assert len(ok) == 1
    i, j, s, failed = ok[0][2]
    assert failed == ([] if fail is None else [1])
    c, _ = synth.config_small(seed=6, n=4000, m=5000)
    ref = oracle.bruteforce(c, t)
    assert len(ref.i) > 0
    compare(i, j, s, ref, t, c.n, csr=c)
