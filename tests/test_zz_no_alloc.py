"""The allocation-free self-join (aps_all_pairs_noalloc) against the allocating one.

Callers that cannot allocate device memory while joining (memory reserved up front by
their own allocator, or a latency-critical thread) pass their own output buffers; the
library takes its scratch from one fixed device array. Two calls in a row must give the
same pairs as aps_all_pairs (the array keeps nothing between calls). This file sorts last
so that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aps():
    import torch

    import paper_1402_3010_gb300 as aps
    from paper_1402_3010_gb300 import _build

    _build.build()
    aps.load()
    torch.cuda.init()
    return aps


def _ref(aps, h):
    p = aps.aps_all_pairs(h)
    try:
        return aps.pairs_to_numpy(p)
    finally:
        aps.aps_pairs_free(p)


@pytest.mark.parametrize("case", ["small", "power_law"])
def test_noalloc_matches_allocating_join_on_two_calls(aps, case):
    import torch

    if case == "small":
        c, t = synth.config_small(seed=1)
    else:
        rng = np.random.default_rng(77)
        lengths = synth.power_law_lengths(rng, 30000, synth.ALPHA_MEAN50, 1, 300)
        c, t = synth.sparse_vectors(30000, 8000, lengths, 1.0, "lognormal", 77, rng=rng), 0.6
    h = aps.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    try:
        ri, rj, rs = _ref(aps, h)
        cap = len(ri) + 100
        i = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        j = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        s = torch.zeros((cap,), dtype=torch.float32, device="cuda")
        for call in range(2):
            n = aps.aps_all_pairs_noalloc(h, i, j, s, torch.cuda.current_stream())
            assert n == len(ri), (call, n, len(ri))
            gi, gj, gs = (a[:n].cpu().numpy() for a in (i, j, s))
            assert np.array_equal(gi, ri) and np.array_equal(gj, rj)
            assert np.abs(gs.astype(np.float64) - rs).max(initial=0.0) <= 1e-5
            keys = gi.astype(np.int64) * c.n + gj
            assert np.all(np.diff(keys) > 0)
            # and the definition itself: the float64 brute force of the oracle
            compare(gi, gj, gs, oracle.bruteforce(c, float(np.float32(t))), float(np.float32(t)), c.n, csr=c)
            st = aps.aps_index_stats(h)
            assert st["pairs"] == n and st["candidates"] >= n
            s.zero_()
    finally:
        aps.aps_index_free(h)


def test_noalloc_allocates_nothing(aps):
    """With the library's allocation-failure hook armed, the allocation-free join still
    succeeds, and the hook is still armed afterwards: the next allocating join fails."""
    import torch

    c, t = synth.config_small(seed=1)
    h = aps.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    try:
        ri, rj, _ = _ref(aps, h)
        out = [torch.empty(len(ri) + 8, dtype=dt, device="cuda") for dt in (torch.int32, torch.int32, torch.float32)]
        aps.aps_debug_fail_alloc(1)
        try:
            n = aps.aps_all_pairs_noalloc(h, *out)
            assert n == len(ri)
            assert np.array_equal(out[0][:n].cpu().numpy(), ri) and np.array_equal(out[1][:n].cpu().numpy(), rj)
            with pytest.raises(aps.APSError) as e:
                p = aps.aps_all_pairs(h)
                aps.aps_pairs_free(p)
            assert e.value.status == aps.ENOMEM
        finally:
            aps.aps_debug_fail_alloc(0)
        p = aps.aps_all_pairs(h)  # disarmed: allocations work again
        assert int(p.count) == len(ri)
        aps.aps_pairs_free(p)
    finally:
        aps.aps_index_free(h)


def test_noalloc_rejects_host_output_arrays_in_the_library(aps):
    """The C entry point itself refuses host memory for its output arrays (callers of the C
    ABI bypass the binding's checks)."""
    import ctypes

    import torch

    c, t = synth.config_small(seed=1)
    h = aps.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    try:
        host = np.zeros(64, np.int32)
        dev = torch.empty(64, dtype=torch.int32, device="cuda")
        cnt = ctypes.c_int64(0)
        lib = aps.load()
        st = lib.aps_all_pairs_noalloc(h, host.ctypes.data, dev.data_ptr(), dev.data_ptr(), 64, ctypes.byref(cnt),
                                       None)
        assert st == aps.EINVAL and "device memory" in aps.aps_last_error()
    finally:
        aps.aps_index_free(h)


def test_noalloc_reports_a_small_capacity_and_oversized_index(aps):
    import torch

    c, t = synth.config_small(seed=1)
    h = aps.aps_build_index(c.indptr, c.idx, c.val, c.n, c.m, t)
    try:
        ri, _, _ = _ref(aps, h)
        assert len(ri) > 1
        small = [torch.empty(1, dtype=dt, device="cuda") for dt in (torch.int32, torch.int32, torch.float32)]
        with pytest.raises(aps.APSError) as e:
            aps.aps_all_pairs_noalloc(h, *small)
        assert e.value.status == aps.EOVERFLOW and e.value.count == len(ri)
    finally:
        aps.aps_index_free(h)
    # 2M one-component vectors: far more (vector, window) slots than the arena holds
    n = 2_000_000
    indptr = np.arange(n + 1, dtype=np.int64)
    idx = (np.arange(n) % 1000).astype(np.int32)
    val = np.ones(n, dtype=np.float32)
    h = aps.aps_build_index(indptr, idx, val, n, 1000, 0.9)
    try:
        out = [torch.empty(16, dtype=dt, device="cuda") for dt in (torch.int32, torch.int32, torch.float32)]
        with pytest.raises(aps.APSError) as e:
            aps.aps_all_pairs_noalloc(h, *out)
        assert e.value.status == aps.EINVAL and "arena" in str(e.value)
    finally:
        aps.aps_index_free(h)
