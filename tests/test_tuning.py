"""Host-side checks of the join's tile-shape table (no GPU work): size buckets, the
default table and its validation."""
import pytest


@pytest.fixture(scope="module")
def A():
    import paper_1402_3010_gb300 as A

    A.load()
    yield A
    A.aps_set_tuning(A.aps_tuning_default(), A.aps_tuning_default(query=True))


def test_size_buckets_follow_their_bounds(A):
    bounds = [b for b in A.TUNE_BOUNDS if b is not None]
    for k, hi in enumerate(bounds):
        assert A.aps_tune_bucket(hi) == k
        assert A.aps_tune_bucket(hi + 1) == k + 1
    assert A.aps_tune_bucket(0) == 0
    assert A.aps_tune_bucket(1 << 40) == A.TUNE_BUCKETS - 1


def test_default_table_is_the_one_window_rule(A):
    """Default: the largest G in {1, 2, 4, 8} whose window of 40960 / G ids holds the
    whole instance, but at least 2 (the rule in force before the table existed)."""
    table = A.aps_tuning_default()
    for n in [1, 100, 512, 513, 2000, 5120, 5121, 9000, 10240, 10241, 20480, 20481, 40960, 40961, 200000]:
        fits = [g for g in (8, 4, 2, 1) if n <= 40960 // g]
        want = max(fits[0] if fits else 1, 2)
        assert table[A.aps_tune_bucket(n)] == want, n


def test_default_queryable_column_equals_the_self_join_column(A):
    """Queries run as (query, window) items, so the queryable column needs no shape of
    its own by default (measured alike on the serving index); it stays settable."""
    assert A.aps_tuning_default(query=True) == A.aps_tuning_default()


def test_set_and_get_round_trip_and_validation(A):
    A.aps_set_tuning([1, 2, 4, 8, 8, 4, 2, 1])
    assert A.aps_get_tuning() == [1, 2, 4, 8, 8, 4, 2, 1]
    for bad in ([3] * 8, [0] * 8, [16] * 8, [8, 8, 8, 8, 4, 2, 2, -1]):
        with pytest.raises(A.APSError) as e:
            A.aps_set_tuning(bad)
        assert e.value.status == A.EINVAL
    assert A.aps_get_tuning() == [1, 2, 4, 8, 8, 4, 2, 1]  # a rejected table changes nothing
    with pytest.raises(ValueError):
        A.aps_set_tuning([8] * 7)
    with pytest.raises(A.APSError):
        A.aps_set_tuning([8] * 8, [3] * 8)  # the queryable column is validated too
    A.aps_set_tuning(A.aps_tuning_default(), A.aps_tuning_default(query=True))
    assert A.aps_get_tuning() == A.aps_tuning_default()
    assert A.aps_get_tuning(query=True) == A.aps_tuning_default(query=True)


def test_autotuner_rejects_bad_batches_before_any_gpu_work(A):
    """Argument checks run on the host before anything touches the device: an empty
    batch, row offsets not starting at 0, m < 1 and t outside (0, 1] are APS_EINVAL,
    and the table in force is unchanged."""
    import numpy as np

    before = A.aps_get_tuning()
    ip = np.array([0, 1, 2], dtype=np.int64)
    ix = np.array([0, 1], dtype=np.int32)
    vv = np.ones(2, dtype=np.float32)
    cases = [
        (np.array([0], dtype=np.int64), [5], [0.5]),          # k = 0
        (np.array([1, 2], dtype=np.int64), [5], [0.5]),       # row_offsets[0] != 0
        (np.array([0, 2], dtype=np.int64), [0], [0.5]),       # m < 1
        (np.array([0, 2], dtype=np.int64), [5], [1.5]),       # t > 1
        (np.array([0, 2], dtype=np.int64), [5], [0.0]),       # t = 0
    ]
    for ro, m, t in cases:
        with pytest.raises(A.APSError) as e:
            A.aps_autotune_batch_csr(ro, ip, ix, vv, np.array(m, np.int32), np.array(t, np.float32))
        assert e.value.status == A.EINVAL
    assert A.aps_get_tuning() == before
