"""The lazy greedy (Algorithm 7's CELF loop) on every launch shape and on both
prefix-extraction paths, against the oracle's naive greedy.

- Cluster shapes: the kernel must cut the pool evaluation by the cluster shape
  it actually received. The selection runs as a plain cooperative launch with
  no cluster attribute and with clusters of 1, 2, 4 and 8 blocks; every shape
  gives the oracle's seeds and sigma*R bit for bit.
- Grid-wide extraction (graphs above 65,536 vertices): the whole seed
  sequence and sigma*R equal the oracle's on a 100,000-vertex graph at two
  values of p, with the work counters showing that prefixes were extracted.
- First-seed gains: mg_v = sum_r |C_r(v)| of every vertex equals the oracle's
  marginal gains for the empty seed set (Algorithm 5, final loop).
- External bulk refresh (by default above 2^20 vertices, forced here): the
  launch stops for the refresh, a streaming launch refreshes the bounds and a
  second launch resumes (refreshes beyond the two queued pairs run inside the
  launch, as without the option). The seeds and sigma*R equal the oracle's,
  at the default refresh threshold and at one evaluation.
"""
import numpy as np
import pytest

import oracle
import paper_2008_03095_gb300 as im
from paper_2008_03095_gb300 import build as im_build
from paper_2008_03095_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    im_build.build()
    im.lib()
    yield
    im.im_debug_clear_overrides()


@pytest.fixture
def clear_overrides():
    im.im_debug_clear_overrides()
    yield
    im.im_debug_clear_overrides()


def _select_async(g, K, R, p, seed):
    import torch

    dev = torch.device("cuda", 0)
    im.im_set_stream(torch.cuda.current_stream())
    ws = im.im_workspace_create(g, R)
    d_seeds = torch.empty(K, dtype=torch.int32, device=dev)
    d_sigma = torch.empty(K, dtype=torch.int64, device=dev)
    im.im_workspace_stats(ws)
    im.im_select_seeds_async(g, ws, K, R, p, seed, d_seeds, d_sigma)
    im.im_workspace_status(ws)
    stats = im.im_workspace_stats(ws)
    seeds = d_seeds.cpu().numpy()
    sigma = d_sigma.cpu().numpy().astype(np.uint64)
    ws.close()
    im.im_set_stream(None)
    return seeds, sigma, stats


# The workload whose selection came out wrong when the cluster shape differed
# from the one the evaluation assumed, plus a larger pool at R = 2048.
SHAPE_CASES = [
    ("powerlaw_n2000", lambda: synth.workload_graph("powerlaw_n2000"), 10, 256, 0.01),
    ("chung_lu_3000_p05", lambda: synth.chung_lu(3000, 15000, 2.2, 11), 25, 2048, 0.05),
]


@pytest.mark.parametrize("shape", [-1, 1, 2, 4, 8])
@pytest.mark.parametrize("name,mk,K,R,p", SHAPE_CASES)
def test_celf_any_cluster_shape_matches_oracle(clear_overrides, shape, name, mk, K, R, p):
    xadj, adj = mk()
    oseeds, osigma = oracle.select_seeds(xadj, adj, K, R, p, 7)
    g = im.im_graph_create(xadj, adj)
    im.im_debug_override(im.IM_OVR_CELF_CLUSTER, shape)
    seeds, sigma, stats = _select_async(g, K, R, p, 7)
    assert stats["check_code"] == 0, stats
    assert np.array_equal(seeds, oseeds), (shape, seeds, oseeds)
    assert np.array_equal(sigma, osigma), (shape, sigma, osigma)
    # the blocking call on the same handle agrees
    bseeds, bsigma = im.im_select_seeds(g, K, R, p, 7)
    assert np.array_equal(bseeds, oseeds) and np.array_equal(bsigma, osigma)
    g.close()


@pytest.fixture(scope="module")
def graph_100k():
    # Chung-Lu, n = 100,000 (above the 65,536 vertices of the block-local
    # extraction), mean degree 10, exponent 2.2
    return synth.chung_lu(100_000, 500_000, 2.2, 17)


@pytest.mark.parametrize("p", [0.01, 0.05])
def test_grid_extraction_path_matches_oracle(graph_100k, p):
    xadj, adj = graph_100k
    K, R, seed = 50, 256, 7
    oseeds, osigma = oracle.select_seeds(xadj, adj, K, R, p, seed)
    g = im.im_graph_create(xadj, adj)
    seeds, sigma, stats = _select_async(g, K, R, p, seed)
    assert stats["check_code"] == 0, stats
    assert stats["celf_extractions"] >= 1
    assert np.array_equal(seeds, oseeds)
    assert np.array_equal(sigma, osigma)
    for shape in (-1, 2):  # the grid path on other launch shapes too
        im.im_debug_override(im.IM_OVR_CELF_CLUSTER, shape)
        try:
            s2, g2 = im.im_select_seeds(g, K, R, p, seed)
        finally:
            im.im_debug_override(im.IM_OVR_CELF_CLUSTER, 0)
        assert np.array_equal(s2, oseeds) and np.array_equal(g2, osigma)
    assert im.im_estimate_spread(g, seeds, R, p, seed) == int(osigma[-1])
    g.close()


@pytest.mark.parametrize("name,mk,R,p", [
    ("powerlaw_n2000", lambda: synth.workload_graph("powerlaw_n2000"), 256, 0.01),
    ("chung_lu_100k", lambda: synth.chung_lu(100_000, 500_000, 2.2, 17), 64, 0.05),
    ("random_300_R33", lambda: synth.random_graph(300, 900, 6), 33, 0.3),
])
def test_first_seed_gains_equal_oracle_marginal_gains(name, mk, R, p):
    xadj, adj = mk()
    lab, siz = oracle.labels(xadj, adj, R, p, 7)
    want = oracle.marginal_gains(lab, siz, np.zeros(0, dtype=np.int32))
    g = im.im_graph_create(xadj, adj)
    got = im.im_debug_first_gains(g, R, p, 7)
    g.close()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("refresh_after,shape", [(0, 0), (1, 0), (1, -1)])
@pytest.mark.parametrize("case", ["local_extraction", "grid_extraction"])
def test_external_refresh_matches_oracle(clear_overrides, graph_100k, case, refresh_after, shape):
    if case == "local_extraction":
        xadj, adj = synth.chung_lu(3000, 15000, 2.2, 11)
        K, R, p = 25, 256, 0.05
    else:
        xadj, adj = graph_100k
        K, R, p = 50, 256, 0.05
    oseeds, osigma = oracle.select_seeds(xadj, adj, K, R, p, 7)
    g = im.im_graph_create(xadj, adj)
    try:
        im.im_debug_override(im.IM_OVR_CELF_EXT_REFRESH, 1)
        im.im_debug_override(im.IM_OVR_CELF_REFRESH_AFTER, refresh_after)
        im.im_debug_override(im.IM_OVR_CELF_CLUSTER, shape)
        seeds, sigma, stats = _select_async(g, K, R, p, 7)
        assert stats["check_code"] == 0, stats
        assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)
        assert stats["celf_refreshes"] >= 1, stats
        im.im_debug_override(im.IM_OVR_CELF_EXT_REFRESH, 2)  # the refresh inside the launch
        s2, g2, st2 = _select_async(g, K, R, p, 7)
        assert st2["celf_refreshes"] == stats["celf_refreshes"]
        assert np.array_equal(s2, oseeds) and np.array_equal(g2, osigma)
    finally:
        g.close()
