"""The dense bench's error report against FP64 (host logic, no GPU): exact inputs report
no error; planted mistakes (a shifted score, a dropped pair, a spurious pair) are caught."""
import sys

import numpy as np

import oracle
import synth


def _bench():
    sys.argv = ["bench.py"]
    import bench

    return bench


def test_exact_pairs_report_no_error():
    b = _bench()
    X = synth.dense_mixture(2000, 64, 20, 0.15, seed=4)
    t = 0.8
    full = oracle.dense_all_pairs(X, t)
    rows = np.random.default_rng(2).choice(2000, 40, replace=False)
    rep = b.dense_precision(X, t, rows, full.i.astype(np.int32), full.j.astype(np.int32),
                            full.s.astype(np.float32), oracle.dense_rows(X, t, rows))
    assert rep["pairs_checked"] > 100
    assert rep["max_abs_err"] < 1e-6
    assert rep["missing_outside_band"] == rep["extra_outside_band"] == 0


def test_planted_mistakes_are_reported():
    b = _bench()
    X = synth.dense_mixture(2000, 64, 20, 0.15, seed=4)
    t = 0.8
    full = oracle.dense_all_pairs(X, t)
    rows = np.random.default_rng(2).choice(2000, 40, replace=False)
    i, j, s = full.i.astype(np.int32), full.j.astype(np.int32), full.s.astype(np.float32).copy()
    touch = np.nonzero(np.isin(i, rows) | np.isin(j, rows))[0]
    far = [k for k in touch.tolist() if abs(float(full.s[k]) - t) > 1e-3]
    s[far[0]] += 1e-4                          # a score off by 1e-4
    keep = np.ones(len(i), bool)
    keep[far[1]] = False                        # a match dropped
    # a non-match added: a sampled row with its least similar other row
    r = int(rows[0])
    X64 = X.astype(np.float64)
    c = int(np.argmin(X64 @ X64[r]))
    a, b2 = min(r, c), max(r, c)
    i2 = np.concatenate([i[keep], [a]]).astype(np.int32)
    j2 = np.concatenate([j[keep], [b2]]).astype(np.int32)
    s2 = np.concatenate([s[keep], [0.9]]).astype(np.float32)
    rep = b.dense_precision(X, t, rows, i2, j2, s2, oracle.dense_rows(X, t, rows))
    assert rep["max_abs_err"] >= 0.9e-4
    assert rep["missing_outside_band"] == 1
    assert rep["extra_outside_band"] == 1
