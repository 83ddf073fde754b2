"""GPU parity of the similarity-graph build (Sec. 2.1 G_S as a CSR adjacency) and of the
k-nn read off it (Sec. 2.2), through the C ABI, against the oracle on the same seeded
pair lists; and the graph of a join result against the graph of the oracle's pairs."""
import numpy as np
import pytest

import oracle
import synth

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


def gpu_graph(aps, i, j, s, n, device=True, flags=0):
    import torch

    if device:
        g = aps.aps_graph_csr(torch.from_numpy(i).cuda(), torch.from_numpy(j).cuda(), torch.from_numpy(s).cuda(), n=n,
                              flags=flags)
    else:
        g = aps.aps_graph_csr(i, j, s, n=n, flags=flags)
    return g


@pytest.mark.parametrize(
    "n,count,skew",
    [(1, 0, 0.0), (2, 1, 0.0), (97, 300, 0.0), (3000, 40000, 1.2), (20000, 400000, 1.0), (5000, 2_000_000, 0.3)],
)
def test_graph_and_knn_match_oracle(aps, n, count, skew):
    i, j, s = synth.pair_list(n, count, seed=11 + n, skew=skew)
    if n == 2:
        i, j, s = np.array([0], np.int32), np.array([1], np.int32), np.array([0.75], np.float32)
    g = gpu_graph(aps, i, j, s, n)
    try:
        rp, col, w = aps.graph_to_numpy(g)
        orp, ocol, ow = oracle.graph_csr(i, j, s, n)
        assert np.array_equal(rp, orp)
        assert np.array_equal(col, ocol)
        assert np.array_equal(w, ow)  # weights are copied, bit for bit
        for k in (1, 7, 64):
            nbr, wk = aps.aps_graph_knn(g, k)
            onbr, owk = oracle.graph_knn(orp, ocol, ow, k)
            assert np.array_equal(nbr, onbr), k
            assert np.array_equal(wk, owk), k
    finally:
        aps.aps_graph_free(g)


def test_knn_ties_and_device_outputs(aps):
    import torch

    n = 600
    i, j, s = synth.pair_list(n, 30000, seed=5, skew=0.7)
    s = (np.round(s * 8) / 8).astype(np.float32)  # many equal weights: ties go to the smaller id
    g = gpu_graph(aps, i, j, s, n, device=False)
    try:
        k = 256
        nb = torch.empty((n, k), dtype=torch.int32, device="cuda")
        wk = torch.empty((n, k), dtype=torch.float32, device="cuda")
        aps.aps_graph_knn(g, k, nb, wk)
        orp, ocol, ow = oracle.graph_csr(i, j, s, n)
        onbr, owk = oracle.graph_knn(orp, ocol, ow, k)
        assert np.array_equal(nb.cpu().numpy(), onbr)
        assert np.array_equal(wk.cpu().numpy(), owk)
    finally:
        aps.aps_graph_free(g)


def test_host_output_graph(aps):
    import paper_1402_3010_gb300 as A

    i, j, s = synth.pair_list(800, 9000, seed=9, skew=0.5)
    g = gpu_graph(aps, i, j, s, 800, flags=A.HOST_OUTPUT)
    try:
        assert g.on_device == 0
        rp, col, w = aps.graph_to_numpy(g)
        orp, ocol, ow = oracle.graph_csr(i, j, s, 800)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(w, ow)
        with pytest.raises(A.APSError):
            aps.aps_graph_knn(g, 3)  # k-nn needs the device graph
    finally:
        aps.aps_graph_free(g)


def test_graph_of_a_join_result(aps):
    """Graph of the library's own join vs the graph of the oracle's pairs (same structure;
    weights within the join's 1e-5)."""
    import torch

    c, _ = synth.config_small(seed=4, n=3000, m=4000)
    t = float(np.float32(0.5))
    ref = oracle.bruteforce(c, t)
    # an input whose scores keep clear of the 1e-5 band, so the pair sets are identical
    assert np.all(np.abs(ref.s - t) > 1e-5)
    ip, ix, vv = (torch.from_numpy(a).cuda() for a in (c.indptr, c.idx, c.val))
    h = aps.aps_build_index(ip, ix, vv, c.n, c.m, t)
    p = aps.aps_all_pairs(h)
    try:
        g = aps.aps_graph_csr(p, n=c.n)
        try:
            rp, col, w = aps.graph_to_numpy(g)
        finally:
            aps.aps_graph_free(g)
    finally:
        aps.aps_pairs_free(p)
        aps.aps_index_free(h)
    orp, ocol, ow = oracle.graph_csr(ref.i, ref.j, ref.s, c.n)
    assert len(col) > 0
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    assert np.abs(w.astype(np.float64) - np.asarray(ow, np.float64)).max() <= 1e-5


@pytest.mark.parametrize("case", ["unsorted", "repeated", "out_of_range", "not_upper"])
def test_malformed_pair_lists_are_rejected(aps, case):
    import paper_1402_3010_gb300 as A

    i = np.array([0, 1, 2, 3], np.int32)
    j = np.array([5, 2, 4, 4], np.int32)
    s = np.ones(4, np.float32) * 0.8
    if case == "unsorted":
        i, j = i[[1, 0, 2, 3]], j[[1, 0, 2, 3]]
    elif case == "repeated":
        i, j = np.array([0, 1, 1, 3], np.int32), np.array([5, 2, 2, 4], np.int32)
    elif case == "out_of_range":
        j = np.array([5, 2, 4, 6], np.int32)
    else:
        i, j = np.array([0, 2, 2, 3], np.int32), np.array([5, 1, 4, 4], np.int32)
    with pytest.raises(A.APSError) as e:
        gpu_graph(aps, i, j, s, 6)
    assert e.value.status == A.EINVAL
