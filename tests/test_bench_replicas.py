"""The multi-GPU bench semantics on CPU: two gloo ranks take the slowest rank's time
(bench.max_over_ranks) and report the whole job's evaluations (bench.replica_value),
the way `bench.py --gpus N` does under torchrun."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0, 25.0, 17.5][rank]
    slowest = bench.max_over_ranks(ms, torch.device("cpu"), world)
    q.put((rank, slowest, bench.replica_value(1000, 3, world, slowest)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert [g[1] for g in got] == [25.0, 25.0]
    # 2 replicas x 1000 evaluations x 3 steps over 25 ms
    assert all(abs(g[2] - 2 * 1000 * 3 / 0.025) < 1e-6 for g in got)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, None, 1) == 12.5
    assert bench.replica_value(500, 4, 1, 20.0) == 500 * 4 / 0.02
