"""GPU parity of the dense path (BF16 tensor-core candidates + exact rescoring) against the
float64 oracle (NumPy X @ X.T + threshold)."""
import numpy as np
import pytest

import oracle
import synth
from parity import compare, dense_dot64

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


def f32(t):
    return float(np.float32(t))


def run_dense(aps, X, t, flags=0, device=True):
    import torch

    Xin = torch.from_numpy(np.ascontiguousarray(X)).cuda() if device else np.ascontiguousarray(X)
    p, st = aps.aps_all_pairs_dense(Xin, t, flags)
    try:
        i, j, s = aps.pairs_to_numpy(p)
    finally:
        aps.aps_pairs_free(p)
    return i, j, s, st


@pytest.mark.parametrize("n,d,k", [(700, 128, 20), (3001, 256, 60), (1500, 64, 30), (1200, 512, 25), (129, 192, 5),
                                   (1100, 512, 25), (257, 384, 6), (5000, 320, 80)])
def test_dense_mixture_full_parity(aps, n, d, k):
    X = synth.dense_mixture(n, d, k, 0.15, seed=n + d)
    t = 0.8
    i, j, s, st = run_dense(aps, X, t)
    ref = oracle.dense_all_pairs(X, f32(t))
    r = compare(i, j, s, ref, f32(t), n, dense=X)
    assert r["pairs"] > 0
    assert st["pairs"] == len(i) and st["candidates"] >= st["pairs"]


def test_dense_many_pairs_near_the_threshold(aps):
    """Random directions in 64-d with t = 0.3: many scores within the BF16 margin of t, so
    the margin and the float32/float64 decisions are exercised."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2500, 64))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X = X.astype(np.float32)
    t = 0.3
    i, j, s, st = run_dense(aps, X, t)
    ref = oracle.dense_all_pairs(X, f32(t))
    compare(i, j, s, ref, f32(t), X.shape[0], dense=X)
    # some reference scores lie just above t: any miss there would fail compare()
    assert np.sum((ref.s >= t) & (ref.s < t + 0.004)) > 10


def test_dense_host_input_and_normalize(aps):
    import paper_1402_3010_gb300 as A

    X = synth.dense_mixture(900, 128, 15, 0.15, seed=9)
    t = 0.85
    ref = oracle.dense_all_pairs(X, f32(t))
    a = run_dense(aps, X, t, device=False)
    compare(a[0], a[1], a[2], ref, f32(t), 900, dense=X)
    b = run_dense(aps, (X * 2.5).astype(np.float32), t, flags=A.NORMALIZE)
    compare(b[0], b[1], b[2], ref, f32(t), 900, tol=2e-5, dense=X)
    with pytest.raises(A.APSError) as e:
        run_dense(aps, (X * 2.5).astype(np.float32), t)
    assert e.value.status == A.EINVAL


@pytest.mark.parametrize("n", [0, 1, 2])
def test_dense_degenerate_sizes(aps, n):
    X = synth.dense_mixture(max(n, 1), 64, 1, 0.0, seed=3)[:n]
    i, j, s, _ = run_dense(aps, X, 0.5)
    assert len(i) == (1 if n == 2 else 0)


def test_dense_bad_arguments(aps):
    import paper_1402_3010_gb300 as A

    X = np.ones((4, 100), np.float32) / 10.0
    with pytest.raises(A.APSError) as e:
        run_dense(aps, X, 0.5)
    assert e.value.status == A.EINVAL


def test_dense_full_size_sampled_rows(aps):
    """The 200k x 256 mixture in the configuration the bench times: rows sampled and
    checked against the float64 oracle one by one."""
    X, t = synth.config_dense()
    i, j, s, st = run_dense(aps, X, t)
    assert st["pairs"] == len(i) > 1_000_000
    keys = i.astype(np.int64) * X.shape[0] + j
    assert np.all(np.diff(keys) > 0) and np.all(i < j)
    rows = np.random.default_rng(1).choice(X.shape[0], 40, replace=False)
    ref = oracle.dense_rows(X, f32(t), rows)
    sel = np.isin(i, rows) | np.isin(j, rows)
    gk = np.unique(keys[sel])
    rk = np.unique(ref.keys(X.shape[0]))
    # outside the 1e-5 band the sets agree
    rmap = dict(zip(ref.keys(X.shape[0]).tolist(), ref.s.tolist()))
    for k in np.setdiff1d(rk, gk).tolist():
        assert abs(rmap[k] - t) <= 1e-5
    smap = dict(zip(keys[sel].tolist(), s[sel].tolist()))
    for k in np.setdiff1d(gk, rk).tolist():  # an extra pair is judged by its float64 score
        a, b = divmod(k, X.shape[0])
        assert abs(dense_dot64(X, a, b) - t) <= 1e-5
    common = np.intersect1d(gk, rk)
    err = max(abs(smap[k] - rmap[k]) for k in common.tolist())
    assert err <= 1e-5


def test_dense_misaligned_device_rows(aps):
    """A device X that is not 16-byte aligned (a view one float into a buffer) gives the
    same pairs."""
    import torch

    X = synth.dense_mixture(1000, 128, 20, 0.15, seed=12)
    t = 0.8
    buf = torch.empty(X.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(X.ravel()).cuda()
    Xm = buf[1:].view(X.shape)
    assert Xm.data_ptr() % 16 != 0
    p, _ = aps.aps_all_pairs_dense(Xm, t)
    try:
        i, j, s = aps.pairs_to_numpy(p)
    finally:
        aps.aps_pairs_free(p)
    compare(i, j, s, oracle.dense_all_pairs(X, f32(t)), f32(t), 1000, dense=X)



@pytest.mark.parametrize("n,d,wait_ns", [(1024, 128, 50_000_000), (40_000, 256, 0)])
def test_dense_wait_limit_expires_and_context_stays_usable(aps, n, d, wait_ns):
    """The tensor-core kernel's bounded waits: with the MMA issuer held back (a release
    that never comes) every pipeline wait runs out, the kernel settles its copies, frees
    tensor memory and returns; the call reports APS_ETIMEOUT within seconds and the next
    join on the same context is exact. At 40k x 256 the TMA ring is full when the waits
    expire; wait_ns = 0 takes the default limit."""
    import time

    import paper_1402_3010_gb300 as A

    X = synth.dense_mixture(n, d, max(30, n // 100), 0.15, seed=n)
    t = 0.8
    before = run_dense(aps, X, t)
    A.aps_debug_dense_stall(1, wait_ns)
    t0 = time.time()
    try:
        with pytest.raises(A.APSError) as e:
            run_dense(aps, X, t)
    finally:
        A.aps_debug_dense_stall(0)
    assert e.value.status == A.ETIMEOUT
    assert time.time() - t0 < 20
    after = run_dense(aps, X, t)
    for a, b in zip(before[:3], after[:3]):
        assert np.array_equal(a, b)
    if n <= 2000:
        ref = oracle.dense_all_pairs(X, f32(t))
        assert compare(after[0], after[1], after[2], ref, f32(t), n, dense=X)["pairs"] > 0


def bf16_round(X):
    """float32 -> the nearest BF16 value (ties to even), as float64 (finite inputs)."""
    b = np.ascontiguousarray(X, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("d", [256, 512])
def test_tensor_products_accumulation_error_within_margin(aps, d):
    """The dense margin delta = (2u + u^2) * 1.002 + 2d * 2^-23 assumes the tensor cores'
    float32 accumulation of the BF16 products errs by at most 2d * 2^-23 on unit rows
    (Sec. 2.1, S = D.D^T). Measured here against the exact (float64) product of the same
    BF16-rounded rows, over every computed entry of a 4096-row mixture with many near-
    duplicate rows (products near 1, the largest sums)."""
    import torch

    n = 4096
    X = synth.dense_mixture(n, d, 64, 0.05, seed=11).astype(np.float32)
    raw = torch.full((n, n), float("nan"), device="cuda")
    aps.aps_dense_tensor_products(torch.from_numpy(X).cuda(), raw)
    S = raw.cpu().numpy().astype(np.float64)
    Xb = bf16_round(X)
    S64 = Xb @ Xb.T
    blk = np.arange(n) // 256
    computed = blk[None, :] >= blk[:, None]
    assert np.isfinite(S[computed]).all() and np.isnan(S[~computed]).all()
    err = np.abs(S[computed] - S64[computed])
    bound = 2 * d * 2.0 ** -23
    assert err.max() <= bound, f"max accumulation error {err.max():.3e} > 2d * 2^-23 = {bound:.3e}"
    # the products are of BF16-rounded rows: their distance to the float32 rows' products is
    # the rounding part of delta, not the accumulation part
    assert np.abs(S64[computed]).max() <= 1.0 + 1e-2
