#!/usr/bin/env python
"""Benchmark of the sparse All-Pairs self-join on one GB300 (or N replicas).

A step is one pass of the whole hot path over the large sparse workload (n = 200,000
vectors, m = 100,000 dimensions, power-law |x| with mean 50 and maximum 2,000, Zipf(1.0)
feature ids, log-normal weights, L2-normalised, t = 0.7): index build from the
device-resident CSR (statistics, dimension ranks, rank-ordered rows, partial-indexing
split, posting lists), the join kernel (probe/accumulate, upperbound, dot(x, y'),
float64 band decisions, compaction) and the output stage that leaves the pairs sorted by
(i, j) in device memory.

Metric: similarity evaluations per second = n(n-1)/2 pairs decided per step / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--t 0.7] [--impl aps|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload (the join
is not sharded across GPUs); the value is all ranks' evaluations / max time.
"""
from __future__ import annotations

import argparse
import copy
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "similarity evaluations/s"
UNIT = "pair-evaluations/s"
WORKLOAD = ("large sparse all-pairs: n=200000, m=100000, |x| power law (alpha=1.4135, mean 50, max 2000), "
            "Zipf(1.0) ids, log-normal(0,1) weights, L2-normalised, FP32")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--t", type=float, default=0.7)
    ap.add_argument("--ranks", type=int, default=2, help="host ranks of --workload horizontal")
    ap.add_argument("--blocks", default="1,2,4", help="dimension block counts of --workload vertical")
    ap.add_argument("--impl", default="aps", choices=["aps", "reference"])
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--m", type=int, default=100_000)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-sample", type=int, default=600, help="queries per core in the oracle's timed sample")
    ap.add_argument("--cpu-cores", type=int, default=0, help="host cores for the CPU baseline (0: all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tiles", default="",
                    help="query groups per size bucket (8 comma-separated values of 1, 2, 4, 8) installed "
                         "before any index is built; default: the library's table")
    ap.add_argument("--query-tiles", default="",
                    help="the same for indexes built to answer queries (the serving index); default: the library's")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched workload: time the default tile table instead of the autotuned one")
    ap.add_argument("--workload", default="sparse",
                    choices=["sparse", "dense", "batched", "serving", "ablation", "graph", "horizontal", "vertical",
                             "split"],
                    help="sparse: the 200k-vector sparse self-join (default line); dense: the 200k x 256 "
                         "embedding self-join on the tensor cores; batched: 512 independent sparse "
                         "instances; serving: query batches against a 1M-vector resident index")
    ap.add_argument("--serve-batches", type=int, default=160)
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: print the sparse headline only, without the dense, batched, serving "
                         "and small-instance records under 'forms'")
    ap.add_argument("--form-steps", type=int, default=5, help="timed steps of each record under 'forms'")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--d", type=int, default=256)
    return ap.parse_args()


def peaks(key="hbm_gbs"):
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d[key]), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}[key], "fallback"


DENSE_WORKLOAD = ("dense embedding all-pairs: n=200000, d=256, 2000-component Gaussian mixture (noise norm 0.15), "
                  "L2-normalised; BF16 tensor-core candidates, FP32/FP64 rescoring")


def workload(n, m, seed=2):
    import synth

    if n == 200_000 and m == 100_000:
        return synth.config_large(seed=seed)
    return synth.config_large(seed=seed, n=n, m=m)


# ------------------------------------------------------------------ clocks sampler
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle baseline
def cpu_baseline(c, t, sample):
    """The oracle's sequential All-Pairs (all-pairs-2 toggles) on a bounded sample: every
    vector is indexed, Find-Matches runs for `sample` random queries. Value = similarity
    evaluations decided by the sampled queries / wall time of the whole call."""
    import oracle

    rng = np.random.default_rng(123)
    mask = np.zeros(c.n, np.uint8)
    mask[rng.choice(c.n, size=min(sample, c.n), replace=False)] = 1
    t0 = time.perf_counter()
    pairs, cnt = oracle.all_pairs(c, float(np.float32(t)), oracle.ALL_PAIRS_2, query_mask=mask)
    dt = time.perf_counter() - t0
    return {
        "value": cnt["evaluations"] / dt,
        "unit": UNIT,
        "cores": 1,
        "kind": "oracle",
        "sample": f"sequential all-pairs-2 (C, FP64) over the full n={c.n} index build, Find-Matches for "
                  f"{int(mask.sum())} random queries ({cnt['evaluations']} evaluations) in {dt:.2f} s",
        "seconds": dt,
    }


def _oracle_worker(job):
    """One host core's share of the CPU baseline (a spawned process): the oracle's
    all-pairs-2 over the full index build with Find-Matches for k random queries."""
    n, m, t, k, seed = job
    sys.path.insert(0, ROOT)
    import oracle

    c = workload(n, m)
    rng = np.random.default_rng(seed)
    mask = np.zeros(c.n, np.uint8)
    mask[rng.choice(c.n, size=min(k, c.n), replace=False)] = 1
    t0 = time.perf_counter()
    _, cnt = oracle.all_pairs(c, float(np.float32(t)), oracle.ALL_PAIRS_2, query_mask=mask)
    return cnt["evaluations"], time.perf_counter() - t0


def host_cores(args) -> int:
    return args.cpu_cores if args.cpu_cores > 0 else (os.cpu_count() or 1)


def cpu_baseline_cores(c, t, per_core: int, cores: int):
    """The oracle on every host core at once (the horizontal idea of Sec. 5.2 on the CPU:
    each core runs the sequential program on its own random queries): value = all cores'
    evaluations / the slowest core's time. A spawned pool (no CUDA state is inherited)."""
    import multiprocessing as mp

    if cores <= 1:
        return cpu_baseline(c, t, per_core)
    jobs = [(c.n, c.m, t, per_core, 1000 + k) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    evals = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    return {
        "value": evals / secs,
        "unit": UNIT,
        "cores": cores,
        "kind": "oracle",
        "sample": f"sequential all-pairs-2 (C, FP64) on each of {cores} host cores at once: each builds the full "
                  f"n={c.n} index and runs Find-Matches for {per_core} random queries ({evals} evaluations in all); "
                  f"slowest core {secs:.2f} s",
        "seconds": secs,
    }


def max_over_ranks(ms: float, dev, world: int) -> float:
    """The slowest rank's time: the job's time for replicas that each did the same work."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    tt = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_value(evals_per_replica: int, steps: int, world: int, ms: float) -> float:
    """Whole-job evaluations/s: every replica's evaluations over the slowest rank's time."""
    return world * evals_per_replica * steps / (ms * 1e-3)


class no_gc:
    """Keep Python's garbage collector out of a timed region (a collection of this process's
    many objects can take tens of milliseconds): collect first, disable, re-enable after."""

    def __enter__(self):
        gc.collect()
        self.was = gc.isenabled()
        gc.disable()

    def __exit__(self, *exc):
        if self.was:
            gc.enable()


def measured_profile(profile: str, source: str, t: float):
    """The committed ncu record of a kernel (profiles/<profile>) when the kernel source is
    byte-identical to the one the counters were taken from, else None."""
    import hashlib

    prof = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        tr = json.load(f)
    with open(os.path.join(ROOT, "paper_1402_3010_gb300", "csrc", source), "rb") as f:
        cur = hashlib.sha1(f.read()).hexdigest()[:16]
    if tr.get("source_sha1_16") == cur and abs(tr.get("t", -1) - t) < 1e-7:
        return tr
    return None


def measured_traffic(profile: str, source: str, t: float):
    """DRAM bytes per launch from a committed ncu capture (profiles/<profile>), valid only
    while the kernel source is byte-identical to the one the counters were taken from."""
    import hashlib

    prof = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        tr = json.load(f)
    with open(os.path.join(ROOT, "paper_1402_3010_gb300", "csrc", source), "rb") as f:
        cur = hashlib.sha1(f.read()).hexdigest()[:16]
    if tr.get("source_sha1_16") == cur and abs(tr.get("t", -1) - t) < 1e-7:
        return tr.get("dram_bytes_per_launch")
    return None


# ------------------------------------------------------------------ the GPU arm
def run_aps(args, rank, world):
    import torch

    import paper_1402_3010_gb300 as aps

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    aps.load()
    t = float(np.float32(args.t))
    c = workload(args.n, args.m)
    stream = torch.cuda.current_stream(dev)
    ip = torch.from_numpy(c.indptr).to(dev)
    ix = torch.from_numpy(c.idx).to(dev)
    vv = torch.from_numpy(c.val).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    evals = c.n * (c.n - 1) // 2

    def step():
        h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t, 0, stream)
        p = aps.aps_all_pairs(h)
        st = aps.aps_index_stats(h)
        cnt = int(p.count)
        aps.aps_pairs_free(p)
        aps.aps_index_free(h)
        return st, cnt

    # warm-up: also sizes the output staging buffers of later steps through the index hint
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        st, cnt = step()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = Clocks(local)
    clocks.start()
    stats = []
    join_ms = []
    l0 = aps.aps_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with no_gc():
        e0.record(stream)
        for _ in range(args.steps):
            flush.fill_(1.0)
            st, cnt = step()
            stats.append(st)
            join_ms.append(st["ms_join"])
        e1.record(stream)
        barrier()
    launches = aps.aps_launch_count() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = max_over_ranks(ms, dev, world)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        time.sleep(3.0)  # let the stopped clock sampler's driver session wind down first
        pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
        hip, hix, hvv = pin(c.indptr), pin(c.idx), pin(c.val)
        npairs = cnt
        oi = torch.empty(npairs, dtype=torch.int32).pin_memory()
        oj = torch.empty(npairs, dtype=torch.int32).pin_memory()
        os_ = torch.empty(npairs, dtype=torch.float32).pin_memory()
        hbytes = c.indptr.nbytes + c.idx.nbytes + c.val.nbytes

        gpu_ms = []

        def e2e_step():
            h = aps.aps_build_index(hip.numpy(), hix.numpy(), hvv.numpy(), c.n, c.m, t, 0, stream)
            p = aps.aps_all_pairs(h)
            n_out = int(p.count)
            if n_out <= npairs:
                aps.aps_pairs_copy_to(p, oi.numpy(), oj.numpy(), os_.numpy(), stream)
            aps.aps_pairs_free(p)
            s_ = aps.aps_index_stats(h)
            gpu_ms.append([round(s_["ms_build"], 2), round(s_["ms_join"], 2), int(s_["reruns"])])
            aps.aps_index_free(h)
            return n_out

        for _ in range(3):
            e2e_step()
        del gpu_ms[:]
        barrier()
        with no_gc():
            t0 = time.perf_counter()
            outs, marks = [], []
            for _ in range(args.e2e_steps):
                outs.append(e2e_step())
                marks.append(time.perf_counter())
            barrier()
            dt = time.perf_counter() - t0
        steps_ms = [round(1e3 * (b - a), 2) for a, b in zip([t0] + marks[:-1], marks)]
        dt = max_over_ranks(dt * 1e3, dev, world) * 1e-3  # the slowest rank's end-to-end time
        e2e = {"value": world * evals * args.e2e_steps / dt, "unit": UNIT, "h2d_bytes_per_step": hbytes,
               "d2h_bytes_per_step": int(max(outs)) * 12, "ms_per_step": 1000 * dt / args.e2e_steps,
               "steps_ms": steps_ms,
               "steps_library_ms": {"fields": ["build", "join (last attempt)", "reruns"], "steps": gpu_ms}}

    if rank != 0:
        return None
    peak, peak_kind = peaks()
    last = stats[-1]
    # algorithmic bytes of one join launch: 8 B per posting entry visited (Alg. 2's adds: an
    # entry after x on one of x's lists, with |y| >= minsize; entries the kernel loads and
    # skips are counted apart, as entries_read), 8 B of (|y'|,
    # maxweight(y')) per candidate, 16 B per dot(x, y') (row pointer + one prefix entry
    # per verified candidate, lower bound) and 8 B per staged output pair
    alg_bytes = 8 * last["visits"] + 8 * last["candidates"] + 16 * last["verified"] + 8 * last["pairs"]
    jm = statistics.mean(join_ms)
    achieved = alg_bytes / (jm * 1e-3) / 1e9
    prof = measured_profile("join_kernel_traffic.json", "join.cu", t) if (c.n, c.m) == (200_000, 100_000) else None
    traffic = prof.get("dram_bytes_per_launch") if prof else None
    line = {
        "metric": METRIC,
        "value": replica_value(evals, args.steps, world, ms),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {
            "workload": WORKLOAD,
            "n": c.n, "m": c.m, "nnz": c.nnz, "t": t,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "256 MB buffer written between steps (L2 flush)",
            "pairs_per_step": cnt,
            "evaluations_per_step": evals,
        },
        "roofline": {
            "bound": "hbm",
            "kernel": "join_kernel",
            "achieved": achieved,
            "peak": peak,
            "unit": "GB/s",
            "frac": achieved / peak,
            "peak_kind": peak_kind + " (hbm_gbs, copy bandwidth)",
            "traffic": traffic,
            "alg_bytes_per_launch": alg_bytes,
            "ms_per_launch": jm,
            # measured DRAM bytes of one launch (ncu, same source) over the launch time, against
            # the same peak; the index is L2-resident, so this is far below the effective figure
            "dram_gbs": traffic / (jm * 1e-3) / 1e9 if traffic else None,
            "dram_frac": traffic / (jm * 1e-3) / 1e9 / peak if traffic else None,
            "bound_by": prof.get("bound_by") if prof else None,
            "counters": prof.get("counters") if prof else None,
        },
        "phases_ms": {"build": last["ms_build"], "join": last["ms_join"], "output": last["ms_sort"],
                      "join_call": last["ms_total"]},
        "work": {k: last[k] for k in ("visits", "candidates", "verified", "pairs", "band", "entries_read")},
        "rates_per_s_of_join": {k: last[k] / (jm * 1e-3) for k in ("visits", "candidates", "pairs")},
        "gpu_launches": launches,
        "e2e": e2e,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_cores(c, t, args.cpu_sample, host_cores(args))
    return line


def run_dense(args, rank, world):
    import torch

    import paper_1402_3010_gb300 as aps
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    aps.load()
    X, t = synth.config_dense(n=args.n, d=args.d)
    t = float(np.float32(t))
    n, d = X.shape
    Xd = torch.from_numpy(X).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    evals = n * (n - 1) // 2

    def step():
        p, st = aps.aps_all_pairs_dense(Xd, t, 0, stream)
        cnt = int(p.count)
        aps.aps_pairs_free(p)
        return st, cnt

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        st, cnt = step()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = Clocks(local)
    clocks.start()
    gemm_ms = []
    l0 = aps.aps_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with no_gc():
        e0.record(stream)
        for _ in range(args.steps):
            flush.fill_(1.0)
            st, cnt = step()
            gemm_ms.append(st["ms_join"])
        e1.record(stream)
        barrier()
    launches = aps.aps_launch_count() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = max_over_ranks(ms, dev, world)
    e2e = None
    if args.e2e_steps > 0:
        hX = torch.from_numpy(X).pin_memory()
        oi = torch.empty(cnt, dtype=torch.int32).pin_memory()
        oj = torch.empty(cnt, dtype=torch.int32).pin_memory()
        os_ = torch.empty(cnt, dtype=torch.float32).pin_memory()

        def e2e_step():
            p, _ = aps.aps_all_pairs_dense(hX.numpy(), t, 0, stream)
            k = int(p.count)
            if k <= cnt:
                aps.aps_pairs_copy_to(p, oi.numpy(), oj.numpy(), os_.numpy(), stream)
            aps.aps_pairs_free(p)
            return k

        e2e_step()
        barrier()
        with no_gc():
            t0 = time.perf_counter()
            outs = [e2e_step() for _ in range(args.e2e_steps)]
            barrier()
            dt = time.perf_counter() - t0
        dt = max_over_ranks(dt * 1e3, dev, world) * 1e-3
        e2e = {"value": world * evals * args.e2e_steps / dt, "unit": UNIT, "h2d_bytes_per_step": X.nbytes,
               "d2h_bytes_per_step": int(max(outs)) * 12, "ms_per_step": 1000 * dt / args.e2e_steps}
    if rank != 0:
        return None
    peak, kind = peaks("bf16_tflops")
    flops = 2.0 * (n * n / 2.0) * d  # n^2 d: the upper triangle of S = X.X^T, diagonal tiles included
    gm = statistics.mean(gemm_ms)
    achieved = flops / (gm * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": replica_value(evals, args.steps, world, ms), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": DENSE_WORKLOAD, "n": n, "d": d, "t": t,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between steps (L2 flush)", "pairs_per_step": cnt,
                   "evaluations_per_step": evals},
        "roofline": {"bound": "tensor", "kernel": "dense_gemm_kernel", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_kind": kind + " (bf16_tflops burst, cuBLAS 8192^3)",
                     "traffic": measured_traffic("dense_gemm_traffic.json", "dense.cu", t) if (n, d) == (200_000, 256)
                     else None,
                     "alg_flops_per_launch": flops, "ms_per_launch": gm},
        "phases_ms": {"gemm": gm, "sort_rescore_compact": st["ms_sort"], "call": st["ms_total"]},
        "work": {k: st[k] for k in ("candidates", "pairs", "band")},
        "gpu_launches": launches, "e2e": e2e, "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        import oracle

        rows = np.random.default_rng(7).choice(n, 2000, replace=False)
        t0 = time.perf_counter()
        ref = oracle.dense_rows(X, t, rows)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(rows) * (n - 1) / dt, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"float64 NumPy X[rows] @ X.T + threshold for 2000 random rows "
                                          f"({len(rows) * (n - 1)} evaluations) in {dt:.2f} s (BLAS threads)"}
        # error against FP64 on the same rows, from one more (untimed) call of the path
        p, _ = aps.aps_all_pairs_dense(Xd, t, 0, stream)
        try:
            gi, gj, gs = aps.pairs_to_numpy(p)
        finally:
            aps.aps_pairs_free(p)
        line["precision_vs_fp64"] = dense_precision(X, t, rows, gi, gj, gs, ref)
        line["accumulation_error"] = dense_accumulation(aps)
    return line


def bf16_round(X):
    """float32 -> the nearest BF16 value (ties to even), as float64 (finite inputs)."""
    b = np.ascontiguousarray(X, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def dense_accumulation(aps, n=4096):
    """The tensor cores' float32 accumulation error, which the dense margin bounds by
    2d * 2^-23: max |S_tc - S_fp64| over every computed entry of a 4096-row mixture (64
    clusters, products up to ~1), S_fp64 the float64 product of the same BF16-rounded rows."""
    import torch

    import synth

    out = {}
    for d in (256, 512):
        X = synth.dense_mixture(n, d, 64, 0.05, seed=11).astype(np.float32)
        raw = torch.full((n, n), float("nan"), device="cuda")
        aps.aps_dense_tensor_products(torch.from_numpy(X).cuda(), raw)
        S = raw.cpu().numpy().astype(np.float64)
        del raw
        Xb = bf16_round(X)
        blk = np.arange(n) // 256
        computed = blk[None, :] >= blk[:, None]
        err = np.abs(S - Xb @ Xb.T)[computed]
        bound = 2 * d * 2.0 ** -23
        out[f"d{d}"] = {"max_abs": float(err.max()), "mean_abs": float(err.mean()), "bound_2d_2^-23": bound,
                        "max_over_bound": float(err.max() / bound), "entries": int(computed.sum())}
    return out


def dense_precision(X, t, rows, gi, gj, gs, ref, band=1e-5):
    """The path's pairs touching `rows` against the float64 scores of the same rows: max and
    mean |score - fp64| over the common pairs, and the pairs one side has and the other lacks,
    split by whether their fp64 score lies within `band` of t (only those may differ)."""
    n = X.shape[0]
    sel = np.isin(gi, rows) | np.isin(gj, rows)
    gk = gi[sel].astype(np.int64) * n + gj[sel]
    g_s = gs[sel].astype(np.float64)
    rk = ref.i.astype(np.int64) * n + ref.j
    rmap = dict(zip(rk.tolist(), np.asarray(ref.s, np.float64).tolist()))
    gmap = dict(zip(gk.tolist(), g_s.tolist()))
    common = [k for k in gmap if k in rmap]
    err = np.array([abs(gmap[k] - rmap[k]) for k in common]) if common else np.zeros(1)
    missing = [rmap[k] for k in rmap if k not in gmap]
    extra = [k for k in gmap if k not in rmap]
    X64 = np.asarray(X, dtype=np.float64)
    extra_fp64 = [float(X64[k // n] @ X64[k % n]) for k in extra]
    m_out = sum(abs(v - t) > band for v in missing)
    e_out = sum(abs(v - t) > band for v in extra_fp64)
    return {"rows": int(len(rows)), "pairs_checked": len(common), "max_abs_err": float(err.max()),
            "mean_abs_err": float(err.mean()), "missing_outside_band": m_out, "missing_in_band": len(missing) - m_out,
            "extra_outside_band": e_out, "extra_in_band": len(extra) - e_out, "band": band}


def sparse_dot64(q, c, a, b):
    """float64 dot product of row a of q with row b of c (sparse rows, sorted ids)."""
    ia, va = q.row(int(a))
    ib, vb = c.row(int(b))
    _, pa, pb = np.intersect1d(ia, ib, assume_unique=True, return_indices=True)
    return float(np.dot(va[pa].astype(np.float64), vb[pb].astype(np.float64)))


def agreement(i, j, s, ref, t, n, dot64, band=1e-5):
    """A result against the oracle's pairs: pairs only one side has, split by whether their
    float64 score (recomputed from the inputs for pairs only the path reports) lies within
    `band` of t (only those may differ), and max |score - fp64| over the common pairs."""
    keys = np.asarray(i, np.int64) * n + np.asarray(j, np.int64)
    rk = ref.keys(n)
    gpu_only = np.setdiff1d(keys, rk)
    ref_only = np.setdiff1d(rk, keys)
    rmap = dict(zip(rk.tolist(), np.asarray(ref.s, np.float64).tolist()))
    missing = [rmap[k] for k in ref_only.tolist()]
    extra = [dot64(*divmod(k, n)) for k in gpu_only.tolist()]
    common = np.intersect1d(keys, rk)
    err = 0.0
    if common.size:
        gs = np.asarray(s, np.float64)[np.searchsorted(keys, common)]
        err = float(np.abs(gs - np.asarray(ref.s, np.float64)[np.searchsorted(rk, common)]).max())
    return {"pairs_checked": int(common.size), "max_abs_err": err,
            "missing_outside_band": int(sum(abs(v - t) > band for v in missing)),
            "missing_in_band": int(sum(abs(v - t) <= band for v in missing)),
            "extra_outside_band": int(sum(abs(v - t) > band for v in extra)),
            "extra_in_band": int(sum(abs(v - t) <= band for v in extra)), "band": band}


BATCHED_WORKLOAD = ("batched sparse all-pairs: 512 independent instances, n log-uniform in [100, 20000], m=50000, "
                    "|x| ~ Poisson(30) in [1,300], Zipf(1.1) ids, U(0,1] weights, t ~ U(0.6, 0.9)")
SERVING_WORKLOAD = ("serving: resident index of 1M sparse vectors (m=200000, power-law |x| mean 40, Zipf(1.0), "
                    "log-normal weights), query batches of log-uniform size 1-4096, t=0.75")


def _sparse_roofline(st, ms):
    peak, kind = peaks()
    alg = 8 * st["visits"] + 8 * st["candidates"] + 16 * st["verified"] + 8 * st["pairs"]
    ach = alg / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "join_kernel", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_kind": kind + " (hbm_gbs, copy bandwidth)", "traffic": None,
            "alg_bytes_per_launch": alg, "ms_per_launch": ms}


def run_batched(args):
    import torch

    import oracle
    import paper_1402_3010_gb300 as aps
    import synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    aps.load()
    ro, c, m, t = synth.config_batched_csr()
    ns = np.diff(ro)
    evals = int((ns * (ns - 1) // 2).sum())
    ip, ix, vv = (torch.from_numpy(a).to(dev) for a in (c.indptr, c.idx, c.val))
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        outs, st = aps.aps_batch_all_pairs_csr(ro, ip, ix, vv, m, t, 0, stream)
        cnt = sum(int(o.count) for o in outs)
        for o in outs:
            aps.aps_pairs_free(o)
        return st, cnt

    # tile shapes per size bucket, chosen by the autotuner on this batch (untimed setup)
    tuned = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        groups, rep = aps.aps_autotune_batch_csr(ro, ip, ix, vv, m, t, 0, stream)
        tuned = {"groups": groups, "default": aps.aps_tuning_default(),
                 "bucket_bounds": [b for b in aps.TUNE_BOUNDS], "seconds": round(time.perf_counter() - t0, 2),
                 "ms_join_default": round(rep["ms_default"], 3), "ms_join_tuned": round(rep["ms_tuned"], 3),
                 "ms_per_group_count": {str(b): rep["ms"][b] for b in range(aps.TUNE_BUCKETS)
                                        if rep["instances"][b] > 0},
                 "instances": rep["instances"], "sampled": rep["sampled"]}
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        st, cnt = step()
    clocks = Clocks(0)
    clocks.start()
    jm = []
    l0 = aps.aps_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    with no_gc():
        e0.record(stream)
        for _ in range(args.steps):
            flush.fill_(1.0)
            st, cnt = step()
            jm.append(st["ms_join"])
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    launches = aps.aps_launch_count() - l0
    clk = clocks.stop()
    line = {
        "metric": METRIC, "value": evals * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": BATCHED_WORKLOAD, "instances": len(ns), "total_n": int(ns.sum()), "nnz": c.nnz,
                   "parallelism": "single GPU", "l2": "256 MB buffer written between steps (L2 flush)",
                   "pairs_per_step": cnt, "evaluations_per_step": evals},
        "roofline": _sparse_roofline(st, statistics.mean(jm)),
        "phases_ms": {"build": st["ms_build"], "join": st["ms_join"], "output": st["ms_sort"],
                      "call": st["ms_total"]},
        "work": {k: st[k] for k in ("visits", "candidates", "verified", "pairs", "band")},
        "gpu_launches": launches, "e2e": None, "clocks": clk,
        "tiles": tuned if tuned is not None else {"groups": aps.aps_get_tuning(), "autotuned": False},
    }
    if not args.no_cpu_baseline:
        sel = np.random.default_rng(11).choice(len(ns), 24, replace=False)
        t0 = time.perf_counter()
        ev = 0
        refs = {}
        for r in sel:
            a, b = int(ro[r]), int(ro[r + 1])
            ip_r = c.indptr[a:b + 1] - c.indptr[a]
            cr = synth.SparseCSR(ip_r, c.idx[c.indptr[a]:c.indptr[b]], c.val[c.indptr[a]:c.indptr[b]], b - a,
                                 int(m[r]))
            refs[int(r)] = (cr, oracle.all_pairs(cr, float(t[r]), oracle.ALL_PAIRS_2)[0])
            ev += (b - a) * (b - a - 1) // 2
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ev / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"sequential all-pairs-2 (C, FP64) on 24 random instances ({ev} "
                                          f"evaluations) in {dt:.2f} s"}
        # the same instances' pairs from one more (untimed) call of the path
        outs, _ = aps.aps_batch_all_pairs_csr(ro, ip, ix, vv, m, t, 0, stream)
        try:
            acc = {"instances": len(refs), "pairs_checked": 0, "max_abs_err": 0.0, "missing_outside_band": 0,
                   "missing_in_band": 0, "extra_outside_band": 0, "extra_in_band": 0, "band": 1e-5}
            for r, (cr, ref) in refs.items():
                gi, gj, gs = aps.pairs_to_numpy(outs[r])
                ag = agreement(gi, gj, gs, ref, float(t[r]), max(cr.n, 1), lambda a, b: sparse_dot64(cr, cr, a, b))
                for k in ("pairs_checked", "missing_outside_band", "missing_in_band", "extra_outside_band",
                          "extra_in_band"):
                    acc[k] += ag[k]
                acc["max_abs_err"] = max(acc["max_abs_err"], ag["max_abs_err"])
        finally:
            for o in outs:
                aps.aps_pairs_free(o)
        line["accuracy"] = acc
    return line


def run_serving(args):
    import torch

    import paper_1402_3010_gb300 as aps
    import synth

    torch.cuda.set_device(0)
    aps.load()
    c, t = synth.config_serving()
    t = float(np.float32(t))
    h = aps.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t, aps.QUERYABLE)
    rng = np.random.default_rng(57)
    sizes = np.clip(np.exp(rng.uniform(0.0, math.log(4096.0), size=args.serve_batches)).astype(np.int64), 1, 4096)
    q = synth.serving_queries(int(sizes.sum()))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    batches = []
    for a, b in zip(offs[:-1], offs[1:]):
        ip = (q.indptr[a:b + 1] - q.indptr[a]).astype(np.int64)
        batches.append((ip, q.idx[q.indptr[a]:q.indptr[b]].copy(), q.val[q.indptr[a]:q.indptr[b]].copy(), int(b - a)))

    overlap = {}

    def run(arrivals):
        """Submit batch k at arrivals[k] seconds (all at once when None); latency = result
        in host memory - arrival."""
        sv = aps.aps_server_create(h, 96 << 30, args.slots)
        lat, pairs = [], 0
        try:
            t0 = time.perf_counter()
            pending = {}
            k = 0
            while k < len(batches) or pending:
                now = time.perf_counter() - t0
                while k < len(batches) and (arrivals is None or arrivals[k] <= now):
                    ip, ix, vv, nq = batches[k]
                    arr = now if arrivals is None else arrivals[k]
                    pending[aps.aps_stream_submit(sv, ip, ix, vv, nq, t)] = arr
                    k += 1
                done = []
                for tk, arr in pending.items():
                    p = aps.aps_stream_poll(sv, tk, 0)
                    if p is not None:
                        lat.append(time.perf_counter() - t0 - arr)
                        pairs += int(p.count)
                        aps.aps_pairs_free(p)
                        done.append(tk)
                for tk in done:
                    del pending[tk]
                if not done:
                    time.sleep(0.0001)
            total = time.perf_counter() - t0
            st = aps.aps_server_timeline(sv)
            overlap.clear()
            overlap.update(st, overlap_frac=st["overlap_ms"] / st["busy_ms"] if st["busy_ms"] > 0 else 0.0)
        finally:
            aps.aps_server_free(sv)
        return total, np.array(lat), pairs

    run(None)  # warm-up
    clocks = Clocks(0)
    clocks.start()
    with no_gc():
        tsat, lsat, pairs = run(None)
    clk = clocks.stop()
    overlap_sat = dict(overlap)
    qps = offs[-1] / tsat
    loads = {}
    for frac in (0.5, 0.8):
        gaps = np.random.default_rng(58).exponential(1.0 / (frac * len(batches) / tsat), size=len(batches))
        with no_gc():
            tt, ll, _ = run(np.cumsum(gaps))
        loads[f"{int(frac * 100)}%"] = {"p50_ms": 1000 * float(np.percentile(ll, 50)),
                                        "p99_ms": 1000 * float(np.percentile(ll, 99)),
                                        "batches_per_s": len(batches) / tt,
                                        "overlap_frac": overlap.get("overlap_frac"),
                                        "max_in_flight": overlap.get("max_in_flight")}
    # the joins' algorithmic bytes: every batch once more through aps_query (untimed), its work
    # counters summed, over the saturated serving time
    work = {"visits": 0, "candidates": 0, "verified": 0, "pairs": 0, "band": 0}
    for ip, ix, vv, nq in batches:
        p = aps.aps_query(h, ip, ix, vv, nq, t)
        aps.aps_pairs_free(p)
        st = aps.aps_index_stats(h)
        for k in work:
            work[k] += int(st[k])
    evals = int(offs[-1]) * c.n
    h2d = sum(ip.nbytes + ix.nbytes + vv.nbytes for ip, ix, vv, _ in batches)
    line = {
        "metric": METRIC, "value": evals / tsat, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1000 * tsat, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": SERVING_WORKLOAD, "index_n": c.n, "index_nnz": c.nnz, "batches": len(batches),
                   "queries": int(offs[-1]), "slots": args.slots, "t": t, "parallelism": "single GPU",
                   "pairs": pairs, "tiles": aps.aps_get_tuning(query=True),
                   "step": "all batches submitted at once and polled to completion (saturated)"},
        "roofline": _sparse_roofline(work, 1000 * tsat),
        "work": work,
        "serving": {"saturated_queries_per_s": qps,
                    "saturated_p50_ms": 1000 * float(np.percentile(lsat, 50)),
                    "saturated_p99_ms": 1000 * float(np.percentile(lsat, 99)), "poisson_load": loads,
                    # device time with two or more batches in flight / device time with any
                    "overlap_frac": overlap_sat.get("overlap_frac"), "device_timeline_ms": overlap_sat},
        "clocks": clk,
        # the serving loop is end to end already: host query CSR in at submit, host pairs out at poll
        "e2e": {"value": evals / tsat, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(pairs) * 12, "ms_per_step": 1000 * tsat},
    }
    line["roofline"]["note"] = ("algorithmic bytes of every batch's join (counters from one untimed pass) over "
                                "the saturated serving time, host submission and polling included")
    if not args.no_cpu_baseline:
        import oracle

        qs_ = batches[0]
        k = min(16, qs_[3])
        sub = synth.SparseCSR(qs_[0][:k + 1].copy(), qs_[1][:qs_[0][k]], qs_[2][:qs_[0][k]], k, c.m)
        t0 = time.perf_counter()
        ref = oracle.bruteforce_cross(sub, c, t)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": k * c.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"float64 brute force (C) of {k} queries against the {c.n}-vector index "
                                          f"({k * c.n} evaluations) in {dt:.2f} s"}
        p = aps.aps_query(h, sub.indptr, sub.idx, sub.val, k, t)
        try:
            gi, gj, gs = aps.pairs_to_numpy(p)
        finally:
            aps.aps_pairs_free(p)
        line["accuracy"] = dict(agreement(gi, gj, gs, ref, t, c.n, lambda a, b: sparse_dot64(sub, c, a, b)),
                                queries=k)
    aps.aps_index_free(h)
    return line


SMALL_WORKLOAD = ("plain sparse all-pairs: n=2000, m=5000, |x| ~ Poisson(20) in [1,200], Zipf(1.1) ids, U(0,1] "
                  "weights, L2-normalised, FP32, t=0.7")


def run_small(args):
    """The 2,000-vector set, a latency case (its 40k components and 320 KB index fit in L2):
    time per call through the C ABI from a device CSR to device pairs (index build + join +
    output), and per join of a built index (its join phase replayed from a CUDA graph)."""
    import torch

    import paper_1402_3010_gb300 as aps
    import synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    aps.load()
    c, t = synth.config_small(seed=1)
    t = float(np.float32(t))
    stream = torch.cuda.current_stream(dev)
    ip, ix, vv = (torch.from_numpy(a).to(dev) for a in (c.indptr, c.idx, c.val))
    evals = c.n * (c.n - 1) // 2
    K = 200

    def call():
        h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t, 0, stream)
        p = aps.aps_all_pairs(h)
        n = int(p.count)
        aps.aps_pairs_free(p)
        st = aps.aps_index_stats(h)
        aps.aps_index_free(h)
        return st, n

    for _ in range(5):
        call()
    clocks = Clocks(0)
    clocks.start()
    lat = []
    l0 = aps.aps_launch_count()
    with no_gc():
        torch.cuda.synchronize(dev)
        for _ in range(K):
            t0 = time.perf_counter()
            st, cnt = call()
            lat.append(1e3 * (time.perf_counter() - t0))
    launches = (aps.aps_launch_count() - l0) / K
    h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t, 0, stream)
    jl, jms = [], []
    with no_gc():
        for _ in range(K):
            t0 = time.perf_counter()
            p = aps.aps_all_pairs(h)
            aps.aps_pairs_free(p)
            jl.append(1e3 * (time.perf_counter() - t0))
            jms.append(aps.aps_index_stats(h)["ms_join"])
    stj = aps.aps_index_stats(h)
    aps.aps_index_free(h)
    clk = clocks.stop()
    ms = statistics.mean(lat)
    rl = _sparse_roofline(stj, statistics.mean(jms))
    rl["bound"] = "latency"
    rl["note"] = "40k components, a 320 KB index: launch and latency bound, the HBM fraction is not the measure"
    line = {
        "metric": METRIC, "value": evals / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": 5,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": SMALL_WORKLOAD, "n": c.n, "m": c.m, "nnz": c.nnz, "t": t, "parallelism": "single GPU",
                   "pairs_per_step": cnt, "evaluations_per_step": evals,
                   "l2": "not flushed: a latency case whose inputs are meant to stay on chip"},
        "latency_ms": {"call_p50": float(np.percentile(lat, 50)), "call_p99": float(np.percentile(lat, 99)),
                       "join_call_p50": float(np.percentile(jl, 50)), "join_call_p99": float(np.percentile(jl, 99)),
                       "join_kernel_mean": statistics.mean(jms)},
        "roofline": rl, "work": {k: stj[k] for k in ("visits", "candidates", "verified", "pairs", "band")},
        "phases_ms": {"build": st["ms_build"], "join": st["ms_join"], "output": st["ms_sort"]},
        "gpu_launches": launches, "gpu_launches_unit": "kernel launches per call", "clocks": clk, "e2e": None,
    }
    if not args.no_cpu_baseline:
        import oracle

        t0 = time.perf_counter()
        oracle.all_pairs(c, t, oracle.ALL_PAIRS_2)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": evals / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"sequential all-pairs-2 (C, FP64) over the whole set in {dt * 1e3:.1f} ms"}
        ref = oracle.bruteforce(c, t)
        p = aps.aps_build_index(ip, ix, vv, c.n, c.m, t, 0, stream)
        try:
            q = aps.aps_all_pairs(p)
            gi, gj, gs = aps.pairs_to_numpy(q)
            aps.aps_pairs_free(q)
        finally:
            aps.aps_index_free(p)
        line["accuracy"] = agreement(gi, gj, gs, ref, t, c.n, lambda a, b: sparse_dot64(c, c, a, b))
    return line


def run_split(args):
    """The vertical algorithm's local pruning inside the join (Sec. 5.1, Lemma 1) on the
    200k-vector workload: the join of the plain kernel next to joins whose costliest
    vectors run as dimension blocks on different CTAs (aps_all_pairs_split), with the pair
    count of each (the tests check the pair sets against the oracle)."""
    import torch

    import paper_1402_3010_gb300 as aps

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    aps.load()
    c = workload(args.n, args.m)
    t = float(np.float32(args.t))
    stream = torch.cuda.current_stream(dev)
    ip, ix, vv = (torch.from_numpy(a).to(dev) for a in (c.indptr, c.idx, c.val))
    h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t, 0, stream)
    steps = max(args.steps, 3)

    def timed(fn):
        fn()  # warm
        join, call, pairs = [], [], 0
        with no_gc():
            for _ in range(steps):
                t0 = time.perf_counter()
                p = fn()
                pairs = int(p.count)
                aps.aps_pairs_free(p)
                call.append(1e3 * (time.perf_counter() - t0))
                join.append(aps.aps_index_stats(h)["ms_join"])
        return statistics.mean(join), statistics.mean(call), pairs

    clocks = Clocks(0)
    clocks.start()
    pj, pc, pp = timed(lambda: aps.aps_all_pairs(h))
    rows = []
    for nblk, heavy in ((2, 200), (4, 200), (2, 2000), (4, 2000)):
        j, cl, pr = timed(lambda: aps.aps_all_pairs_split(h, nblk, heavy))
        rows.append({"blocks": nblk, "heavy_vectors": heavy, "join_kernel_ms": round(j, 3), "call_ms": round(cl, 3),
                     "pairs": pr, "same_count_as_plain": pr == pp})
    clk = clocks.stop()
    aps.aps_index_free(h)
    evals = c.n * (c.n - 1) // 2
    return {
        "metric": METRIC, "value": evals / (pc * 1e-3), "unit": UNIT, "ms_per_step": pc, "steps": steps,
        "dtype": "f32",
        "config": {"workload": "the vertical algorithm's local pruning inside the join, on " + WORKLOAD,
                   "n": c.n, "m": c.m, "t": t, "step": "one join call of the built index"},
        "split": {"plain_join_kernel_ms": round(pj, 3), "plain_call_ms": round(pc, 3), "plain_pairs": pp,
                  "runs": rows,
                  "note": "call_ms includes the merge of the blocks' pairs (sort, first occurrences, placement)"},
        "clocks": clk,
    }


FORM_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "dtype", "config", "roofline", "latency_ms", "split",
             "phases_ms", "work", "serving", "tiles", "clocks", "cpu_baseline", "accuracy", "precision_vs_fp64",
             "accumulation_error", "e2e", "gpu_launches", "gpu_launches_unit")


def as_form(line):
    """A full bench line as a record under the headline's 'forms'."""
    return {k: line[k] for k in FORM_KEYS if k in line and line[k] is not None}


def run_forms(args):
    """The dense, batched, serving and small-instance forms measured beside the headline, on
    the same GPU in the same run (each with its own clocks, roofline, oracle baseline and
    accuracy against the oracle)."""
    a = copy.copy(args)
    a.steps, a.warmup, a.e2e_steps = args.form_steps, 3, 2
    forms = {}
    for name, fn in (("small", lambda: run_small(a)), ("dense", lambda: run_dense(a, 0, 1)),
                     ("batched", lambda: run_batched(a)), ("serving", lambda: run_serving(a)),
                     ("split", lambda: run_split(a))):
        t0 = time.perf_counter()
        rec = as_form(fn())
        rec["seconds"] = round(time.perf_counter() - t0, 1)
        forms[name] = rec
        gc.collect()
    return forms


def run_reference(args, rank):
    """The reference arm: the CPU oracle (no upstream implementation exists), on rank 0."""
    if rank != 0:
        return None
    t = float(np.float32(args.t))
    c = workload(args.n, args.m)
    secs = 0.0
    cores = host_cores(args)
    for _ in range(max(args.warmup, 0)):
        cpu_baseline_cores(c, t, max(args.cpu_sample // 8, 10), cores)
    res = []
    for _ in range(args.steps):
        r = cpu_baseline_cores(c, t, args.cpu_sample, cores)
        res.append(r)
        secs += r["seconds"]
    value = statistics.mean(r["value"] for r in res)
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000 * secs / max(args.steps, 1),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": WORKLOAD, "n": c.n, "m": c.m, "nnz": c.nnz, "t": t,
                   "parallelism": f"CPU, {cores} host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": res[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_ablation(args, rank, world):
    """The paper's optimisation-variant matrix (Sec. 4, Tables 2-3) on the sparse workload:
    each variant's index build + join, timed, with its work counters, and its pairs checked
    against all-pairs-2's (identical keys, scores within 1e-5). Rank 0 only."""
    import torch

    import paper_1402_3010_gb300 as aps

    if rank != 0:
        return None
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    aps.load()
    t = float(np.float32(args.t))
    c = workload(args.n, args.m)
    stream = torch.cuda.current_stream(dev)
    ip = torch.from_numpy(c.indptr).to(dev)
    ix = torch.from_numpy(c.idx).to(dev)
    vv = torch.from_numpy(c.val).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    evals = c.n * (c.n - 1) // 2
    order = ["all-pairs-2", "all-pairs-0-array", "all-pairs-0-remscore", "all-pairs-0-minsize", "all-pairs-1-array",
             "all-pairs-1-remscore", "all-pairs-1-upperbound", "all-pairs-1-minsize", "all-pairs-1-remscore-minsize"]
    ref = None
    rows = []
    clocks = Clocks(dev.index or 0)
    clocks.start()
    for name in order:
        flags = aps.VARIANTS[name]

        def step(keep=False):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            flush.fill_(1.0)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t, flags, stream)
            p = aps.aps_all_pairs(h)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            st = aps.aps_index_stats(h)
            out = aps.pairs_to_numpy(p) if keep else None
            aps.aps_pairs_free(p)
            aps.aps_index_free(h)
            return e0.elapsed_time(e1), st, out

        step()  # warm-up (sizes the staging buffer)
        times = []
        for k in range(max(args.steps, 1)):
            ms, st, out = step(keep=(k == 0))
            times.append(ms)
        i, j, s = out
        keys = i.astype(np.int64) * c.n + j
        if ref is None:
            ref = (keys, s)
            same, ds = True, 0.0
        else:
            same = bool(np.array_equal(keys, ref[0]))
            ds = float(np.abs(s - ref[1]).max(initial=0.0)) if same else None
        ms = statistics.median(times)
        rows.append({"variant": name, "flags": flags, "ms_step": ms, "ms_build": st["ms_build"],
                     "ms_join": st["ms_join"], "evaluations_per_s": evals / (ms * 1e-3),
                     "visits": st["visits"], "candidates": st["candidates"], "verified": st["verified"],
                     "pairs": st["pairs"], "band": st["band"], "same_pairs_as_all_pairs_2": same,
                     "max_score_diff": ds})
    clk = clocks.stop()
    base = rows[0]
    return {
        "metric": METRIC,
        "value": base["evaluations_per_s"],
        "unit": UNIT,
        "n_gpus": 1,
        "steps": max(args.steps, 1),
        "warmup": 1,
        "ms_per_step": base["ms_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": "optimisation-variant matrix (paper Sec. 4, Tables 2-3) on " + WORKLOAD,
                   "n": c.n, "m": c.m, "nnz": c.nnz, "t": t, "parallelism": "single GPU",
                   "l2": "256 MB buffer written before each step (L2 flush)"},
        "variants": rows,
        "clocks": clk,
    }


def run_graph(args, rank, world):
    """The similarity graph G_S (Sec. 2.1) of the sparse workload's join result: CSR build
    from the device pair list and k-nn (k = 16, Sec. 2.2), timed with CUDA events over
    --steps repetitions (the join itself is untimed here). Rank 0 only."""
    import torch

    import paper_1402_3010_gb300 as aps

    if rank != 0:
        return None
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    aps.load()
    t = float(np.float32(args.t))
    c = workload(args.n, args.m)
    stream = torch.cuda.current_stream(dev)
    ip, ix, vv = (torch.from_numpy(a).to(dev) for a in (c.indptr, c.idx, c.val))
    h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t, 0, stream)
    p = aps.aps_all_pairs(h)
    aps.aps_index_free(h)
    npairs = int(p.count)
    k = 16
    nbr = torch.empty((c.n, k), dtype=torch.int32, device=dev)
    wk = torch.empty((c.n, k), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        flush.fill_(1.0)
        e0.record(stream)
        g = aps.aps_graph_csr(p, n=c.n, stream=stream)
        e1.record(stream)
        aps.aps_graph_knn(g, k, nbr, wk, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        nnz = int(g.nnz)
        aps.aps_graph_free(g)
        return e0.elapsed_time(e1), e1.elapsed_time(e2), nnz

    for _ in range(max(args.warmup, 3)):
        step()
    clocks = Clocks(dev.index or 0)
    clocks.start()
    l0 = aps.aps_launch_count()
    res = [step() for _ in range(args.steps)]
    launches = aps.aps_launch_count() - l0
    clk = clocks.stop()
    aps.aps_pairs_free(p)
    csr_ms = statistics.median(r[0] for r in res)
    knn_ms = statistics.median(r[1] for r in res)
    peak, peak_kind = peaks()
    # algorithmic bytes of the CSR build: read the pair list once (12 B/pair), write both
    # adjacency entries (2 x 8 B/pair) and row_ptr (8 B/vertex)
    alg = 28 * npairs + 8 * (c.n + 1)
    achieved = alg / (csr_ms * 1e-3) / 1e9
    return {
        "metric": "similarity-graph edges/s",
        "value": npairs / (csr_ms * 1e-3),
        "unit": "undirected edges/s (CSR build)",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": csr_ms + knn_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32/f32",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": "similarity graph G_S (CSR adjacency + k-nn, k=16) of " + WORKLOAD,
                   "n": c.n, "m": c.m, "t": t, "edges": npairs, "adjacency_entries": 2 * npairs,
                   "parallelism": "single GPU", "l2": "256 MB buffer written before each step (L2 flush)"},
        "phases_ms": {"csr": csr_ms, "knn16": knn_ms},
        "roofline": {"bound": "hbm", "kernel": "graph CSR build (counts, scans, j-sort, fills)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind + " (hbm_gbs, copy bandwidth)", "traffic": None,
                     "alg_bytes_per_launch": alg, "ms_per_launch": csr_ms},
        "gpu_launches": launches,
        "clocks": clk,
    }


def _horizontal_rank(rank, p, port, n, m, t, out_q):
    """One host rank of --workload horizontal (a spawned process)."""
    from datetime import timedelta

    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_1402_3010_gb300 import horizontal as H

    torch.cuda.set_device(rank % max(torch.cuda.device_count(), 1))
    c = workload(n, m)
    store = dist.TCPStore("127.0.0.1", port, p, rank == 0, timedelta(seconds=900))
    part_of = lambda r: H.cyclic_part(c.indptr, c.idx, c.val, c.m, r, p)  # noqa: E731
    matcher = H.GpuMatcher()
    store.set(f"ready/{rank}", b"1")
    store.wait([f"ready/{r}" for r in range(p)])
    t0 = time.perf_counter()
    res = H.horizontal_all_pairs(rank, p, store, part_of, t, matcher, timeout_s=900.0)
    dt = time.perf_counter() - t0
    info = {"rank": rank, "seconds": dt, "part_bytes": int(part_of(rank).indptr.nbytes + part_of(rank).idx.nbytes
                                                           + part_of(rank).val.nbytes)}
    if res is not None:
        i, j, s_, failed = res
        info.update(pairs=int(i.size), keysum=int((i.astype(np.int64) * n + j).sum() % (1 << 61)), failed=failed)
    out_q.put(info)


def run_horizontal(args, rank, world):
    """The horizontal driver (Sec. 5.2, Alg. 6) with --ranks host processes
    on this machine's GPU(s), against the single-process join of the same workload."""
    import multiprocessing as mp
    import socket

    import torch

    import paper_1402_3010_gb300 as aps

    if rank != 0:
        return None
    aps.load()
    t = float(np.float32(args.t))
    c = workload(args.n, args.m)
    dev = torch.device("cuda", 0)
    ip, ix, vv = (torch.from_numpy(a).to(dev) for a in (c.indptr, c.idx, c.val))
    h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t)
    pr = aps.aps_all_pairs(h)
    i, j, _ = aps.pairs_to_numpy(pr)
    aps.aps_pairs_free(pr)
    aps.aps_index_free(h)
    ref_pairs, ref_sum = int(i.size), int((i.astype(np.int64) * c.n + j).sum() % (1 << 61))
    del ip, ix, vv
    torch.cuda.empty_cache()
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = args.ranks
    procs = [ctx.Process(target=_horizontal_rank, args=(r, p, port, args.n, args.m, t, q)) for r in range(p)]
    for x in procs:
        x.start()
    infos = []
    deadline = time.time() + 1200
    while len(infos) < p and time.time() < deadline:
        try:
            infos.append(q.get(timeout=5))
        except Exception:
            if not any(x.is_alive() for x in procs):  # every rank exited: nothing more will come
                break
    for x in procs:
        x.join(30)
        if x.is_alive():
            x.kill()
    if len(infos) < p:
        return {"metric": METRIC, "value": None, "unit": UNIT,
                "error": f"{p - len(infos)} of {p} ranks returned nothing"}
    secs = max(x["seconds"] for x in infos)
    root = [x for x in infos if x["rank"] == 0][0]
    part_bytes = {x["rank"]: x["part_bytes"] for x in infos}
    exchanged = sum(part_bytes[a] for b in range(p) for a in range(b))
    evals = c.n * (c.n - 1) // 2
    return {
        "metric": METRIC,
        "value": evals / secs,
        "unit": UNIT,
        "n_gpus": max(torch.cuda.device_count(), 1),
        "steps": 1,
        "warmup": 0,
        "ms_per_step": 1000 * secs,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": f"horizontal driver (Sec. 5.2, Alg. 6), {p} host ranks, on " + WORKLOAD,
                   "n": c.n, "m": c.m, "t": t, "parallelism": f"{p} host processes, vector-partitioned (cyclic)",
                   "exchange": "TCPStore key-value store on 127.0.0.1"},
        "horizontal": {"ranks": p, "wall_s_per_rank": {x["rank"]: x["seconds"] for x in infos},
                       "pairs": root["pairs"], "same_pairs_as_single_process": root["pairs"] == ref_pairs
                       and root["keysum"] == ref_sum, "failed_ranks": root["failed"],
                       "vector_bytes_exchanged": exchanged},
    }


def run_vertical(args, rank, world):
    """The vertical algorithm with local pruning (Sec. 5.1, Lemma 1, Eq. 2) for
    each block count in --blocks: p block joins at t/p on the GPU, the union completed
    exactly (aps_pairs_verify), checked against the plain join of the same workload."""
    import torch

    import paper_1402_3010_gb300 as aps
    from paper_1402_3010_gb300 import vertical as V

    if rank != 0:
        return None
    aps.load()
    t = float(np.float32(args.t))
    c = workload(args.n, args.m)
    dev = torch.device("cuda", 0)
    ip, ix, vv = (torch.from_numpy(a).to(dev) for a in (c.indptr, c.idx, c.val))
    h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t)
    pr = aps.aps_all_pairs(h)
    i, j, _ = aps.pairs_to_numpy(pr)
    aps.aps_pairs_free(pr)
    aps.aps_index_free(h)
    ref = (int(i.size), int((i.astype(np.int64) * c.n + j).sum() % (1 << 61)))
    rows = []
    for p in [int(x) for x in args.blocks.split(",")]:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out, info = V.vertical_all_pairs(c.indptr, c.idx, c.val, c.n, c.m, t, p)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        a, b, _ = aps.pairs_to_numpy(out)
        aps.aps_pairs_free(out)
        got = (int(a.size), int((a.astype(np.int64) * c.n + b).sum() % (1 << 61)))
        rows.append({"blocks": p, "t_local": info["t_local"], "seconds": dt, "local_pairs": info["local_pairs"],
                     "candidates": info["candidates"], "pairs": got[0], "same_pairs_as_join": got == ref})
    evals = c.n * (c.n - 1) // 2
    best = min(rows, key=lambda r: r["seconds"])
    return {
        "metric": METRIC, "value": evals / best["seconds"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": 1000 * best["seconds"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64", "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": "vertical algorithm with local pruning (Sec. 5.1) on " + WORKLOAD, "n": c.n, "m": c.m,
                   "t": t, "parallelism": "dimension blocks joined in turn on one GPU",
                   "timing": "wall clock of the whole call (host projection included)"},
        "vertical": rows,
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if (args.tiles or args.query_tiles) and args.impl != "reference":
        import paper_1402_3010_gb300 as aps

        aps.load()
        cols = [[int(v) for v in a.split(",")] if a else None for a in (args.tiles, args.query_tiles)]
        aps.aps_set_tuning(cols[0] or aps.aps_get_tuning(), cols[1])
    if args.impl == "reference":
        line = run_reference(args, rank)
    elif args.workload == "dense":
        line = run_dense(args, rank, world)
    elif args.workload == "batched":
        line = run_batched(args)
    elif args.workload == "serving":
        line = run_serving(args)
    elif args.workload == "ablation":
        line = run_ablation(args, rank, world)
    elif args.workload == "graph":
        line = run_graph(args, rank, world)
    elif args.workload == "horizontal":
        line = run_horizontal(args, rank, world)
    elif args.workload == "vertical":
        line = run_vertical(args, rank, world)
    elif args.workload == "split":
        line = run_split(args)
    else:
        line = run_aps(args, rank, world)
        if line is not None and world == 1 and not args.no_forms and args.workload == "sparse":
            line["forms"] = run_forms(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "aps":
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
