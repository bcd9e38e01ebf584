"""Parity of the sm_103a path (through the C ABI) with the CPU oracle.

Everything the method computes is integer and exact, so every comparison is
bit-exact: per-sample random values, edge hashes, component labels, the size
memo, the seed sequence and sigma*R."""
import numpy as np
import pytest

import oracle
import paper_2008_03095_gb300 as im
from paper_2008_03095_gb300 import build as im_build
from paper_2008_03095_gb300 import synth
from tests import _util

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    im_build.build()
    im.lib()


def _graph(xadj, adj):
    return im.im_graph_create(xadj, adj)


# ------------------------------------------------------------------ primitives


@pytest.mark.parametrize("seed", [7, 5489, 0xFFFFFFFF, 0])
@pytest.mark.parametrize("R", [1, 623, 624, 625, 1024, 2048, 5000])
def test_lane_randoms_equal_mt19937(seed, R):
    assert np.array_equal(im.im_debug_lane_randoms(R, seed), oracle.mt19937(seed, R))


def test_lane_randoms_standard_value_and_max_R():
    (seed, idx, val), = [tuple(int(t) for t in row)
                         for row in _util.golden_lines("mt19937_standard.txt")]
    assert int(im.im_debug_lane_randoms(idx, seed)[-1]) == val
    assert np.array_equal(im.im_debug_lane_randoms(65536, 3), oracle.mt19937(3, 65536))


def test_edge_hash_equals_oracle():
    rng = np.random.default_rng(1)
    u = rng.integers(0, 2 ** 31 - 1, size=4000).astype(np.int32)
    v = rng.integers(0, 2 ** 31 - 1, size=4000).astype(np.int32)
    u[:50] = v[:50]  # self pairs
    u[50:100] = np.arange(50)
    v[50:100] = np.arange(50)[::-1]
    got = im.im_debug_edge_hash(u, v)
    want = np.array([oracle.edge_hash(int(a), int(b)) for a, b in zip(u, v)], dtype=np.uint32)
    assert np.array_equal(got, want)
    assert np.array_equal(got, im.im_debug_edge_hash(v, u))


# ------------------------------------------------------------------ small graphs

SMALL = [
    ("chung_lu_500", lambda: synth.chung_lu(500, 2000, 2.3, 5)),
    ("random_300", lambda: synth.random_graph(300, 900, 6)),
    ("chung_lu_1200_hub", lambda: synth.chung_lu(1200, 6000, 2.1, 9)),
]


@pytest.mark.parametrize("name,mk", SMALL)
@pytest.mark.parametrize("R", [1, 33, 256])
@pytest.mark.parametrize("p", [0.0, 0.01, 0.1, 0.5, 1.0])
def test_tables_parity_small(name, mk, R, p):
    xadj, adj = mk()
    g = _graph(xadj, adj)
    lab, siz = oracle.labels(xadj, adj, R, p, 7)
    assert np.array_equal(im.im_debug_labels(g, R, p, 7), lab)
    assert np.array_equal(im.im_debug_sizes(g, R, p, 7), siz)


@pytest.mark.parametrize("name,mk", SMALL)
@pytest.mark.parametrize("R,p", [(1, 0.3), (33, 0.05), (256, 0.01), (256, 0.1), (64, 0.0),
                                 (64, 1.0), (100, 0.5)])
def test_select_and_spread_parity_small(name, mk, R, p):
    xadj, adj = mk()
    n = xadj.shape[0] - 1
    g = _graph(xadj, adj)
    K = min(25, n)
    seeds, sigma = im.im_select_seeds(g, K, R, p, 11)
    oseeds, osigma = oracle.select_seeds(xadj, adj, K, R, p, 11)
    assert np.array_equal(seeds, oseeds)
    assert np.array_equal(sigma, osigma)
    assert im.im_estimate_spread(g, seeds, R, p, 11) == int(sigma[-1])
    rng = np.random.default_rng(R)
    S = rng.integers(0, n, size=7)
    S[3] = S[1]  # duplicate seeds count once
    assert im.im_estimate_spread(g, S, R, p, 11) == oracle.estimate_spread(xadj, adj, S, R, p, 11)


def test_select_all_vertices_and_tiny_graphs():
    xadj, adj = synth.random_graph(40, 60, 3)
    g = _graph(xadj, adj)
    for R, p in ((5, 0.2), (64, 0.6), (3, 1.0)):
        seeds, sigma = im.im_select_seeds(g, 40, R, p, 2)
        oseeds, osigma = oracle.select_seeds(xadj, adj, 40, R, p, 2)
        assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)
        assert sorted(seeds.tolist()) == list(range(40))
        assert int(sigma[-1]) == 40 * R
    # single vertex, no edges
    g1 = _graph(np.array([0, 0], dtype=np.int32), np.array([], dtype=np.int32))
    s, sg = im.im_select_seeds(g1, 1, 17, 0.5, 1)
    assert s.tolist() == [0] and sg.tolist() == [17]
    assert im.im_estimate_spread(g1, [0, 0], 17, 0.5, 1) == 17
    assert im.im_estimate_spread(g1, [], 17, 0.5, 1) == 0
    s0, sg0 = im.im_select_seeds(g1, 0, 17, 0.5, 1)
    assert s0.shape == (0,)


def test_isolated_vertices_self_loops_duplicates_unsorted():
    n = 60
    rng = np.random.default_rng(8)
    e = [(int(a), int(b)) for a, b in rng.integers(0, 40, size=(120, 2))]  # 40..59 isolated
    e += [(5, 5), (7, 7)]  # self-loops (both orientations: two arcs u->u)
    e += e[:10]  # duplicates
    u = np.array([a for a, b in e] + [b for a, b in e])
    v = np.array([b for a, b in e] + [a for a, b in e])
    order = rng.permutation(len(u))  # unsorted neighbour lists
    u, v = u[order], v[order]
    idx = np.argsort(u, kind="stable")
    adj = v[idx].astype(np.int32)
    xadj = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(u, minlength=n), out=xadj[1:])
    assert oracle.validate_csr(xadj, adj)
    g = _graph(xadj, adj)
    for R, p in ((32, 0.2), (7, 0.7), (50, 1.0)):
        lab, siz = oracle.labels(xadj, adj, R, p, 4)
        assert np.array_equal(im.im_debug_labels(g, R, p, 4), lab)
        assert np.array_equal(im.im_debug_sizes(g, R, p, 4), siz)
        seeds, sigma = im.im_select_seeds(g, 20, R, p, 4)
        oseeds, osigma = oracle.select_seeds(xadj, adj, 20, R, p, 4)
        assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)


# ------------------------------------------------------------------ worked example, brute force


def test_worked_example_figures_3_4_on_gpu():
    xadj, adj, mask, exp = _util.worked_example()
    g = _graph(xadj, adj)
    seeds, sigma, lab, siz = im.im_debug_select_seeds_masked(g, 1, mask, tables=True)
    assert np.array_equal(lab, exp["labels"])
    olab, osiz = oracle.labels_masked(xadj, adj, mask)
    assert np.array_equal(siz, osiz)
    assert int(seeds[0]) == exp["first_seed"] and int(sigma[0]) == exp["first_sigmaR"]
    seeds5, sigma5 = im.im_debug_select_seeds_masked(g, 5, mask)
    oseeds5, osigma5 = oracle.select_seeds_masked(xadj, adj, 5, mask)
    assert np.array_equal(seeds5, oseeds5) and np.array_equal(sigma5, osigma5)
    assert im.im_debug_estimate_spread_masked(g, [0], mask) == 9


def test_all_live_subsets_masks_on_gpu():
    edges = [(0, 1), (1, 2), (2, 3), (0, 3), (1, 4), (4, 5), (5, 6), (2, 6), (6, 7), (0, 7)]
    xadj, adj = synth.csr_from_edges(8, [a for a, b in edges], [b for a, b in edges])
    R = 2 ** len(edges)
    idx = {e: i for i, e in enumerate(edges)}
    mask = _util.arc_mask(xadj, adj, lambda u, v, r: (r >> idx[tuple(sorted((u, v)))]) & 1, R)
    g = _graph(xadj, adj)
    seeds, sigma, lab, siz = im.im_debug_select_seeds_masked(g, 8, mask, tables=True)
    olab, osiz = oracle.labels_masked(xadj, adj, mask)
    assert np.array_equal(lab, olab) and np.array_equal(siz, osiz)
    oseeds, osigma = oracle.select_seeds_masked(xadj, adj, 8, mask)
    assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)
    for S in ([0], [3, 5], [1, 6, 7, 1]):
        assert (im.im_debug_estimate_spread_masked(g, S, mask) ==
                oracle.estimate_spread_masked(xadj, adj, S, mask))


# ------------------------------------------------------------------ workloads


@pytest.fixture(scope="module")
def g2000():
    xadj, adj = synth.workload_graph("powerlaw_n2000")
    return xadj, adj, _graph(xadj, adj)


def test_workload_n2000_full_parity(g2000):
    xadj, adj, g = g2000
    w = synth.WORKLOADS["powerlaw_n2000"]
    R, K, s = w["R"], w["K"], w["rng_seed"]
    for p in w["ps"] + (0.05,):
        lab, siz = oracle.labels(xadj, adj, R, p, s)
        assert np.array_equal(im.im_debug_labels(g, R, p, s), lab)
        assert np.array_equal(im.im_debug_sizes(g, R, p, s), siz)
        seeds, sigma = im.im_select_seeds(g, K, R, p, s)
        oseeds, osigma = oracle.greedy_from_tables(lab, siz, K)
        assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)
        assert im.im_estimate_spread(g, seeds, R, p, s) == int(sigma[-1])


@pytest.fixture(scope="module")
def g15233():
    xadj, adj = synth.workload_graph("powerlaw_n15233")
    return xadj, adj, _graph(xadj, adj)


@pytest.mark.parametrize("p", [0.005, 0.01, 0.05])
def test_workload_n15233_full_parity(g15233, p):
    xadj, adj, g = g15233
    w = synth.WORKLOADS["powerlaw_n15233"]
    R, K, s = w["R"], w["K"], w["rng_seed"]
    lab, siz = oracle.labels(xadj, adj, R, p, s)
    assert np.array_equal(im.im_debug_labels(g, R, p, s), lab)
    assert np.array_equal(im.im_debug_sizes(g, R, p, s), siz)
    seeds, sigma = im.im_select_seeds(g, K, R, p, s)
    oseeds, osigma = oracle.greedy_from_tables(lab, siz, K)
    assert np.array_equal(seeds, oseeds)
    assert np.array_equal(sigma, osigma)
    spread = im.im_estimate_spread(g, seeds, R, p, s)
    assert spread == int(sigma[-1])
    assert spread == oracle.estimate_spread(xadj, adj, seeds, R, p, s)


def test_repeated_runs_are_identical(g15233):
    xadj, adj, g = g15233
    a = im.im_select_seeds(g, 50, 1024, 0.01, 3)
    for _ in range(3):
        b = im.im_select_seeds(g, 50, 1024, 0.01, 3)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_async_api_on_torch_stream_matches_blocking(g15233):
    torch = pytest.importorskip("torch")
    xadj, adj, g = g15233
    ws = im.im_workspace_create(g, 1024)
    stream = torch.cuda.Stream()
    im.im_set_stream(stream)
    try:
        d_seeds = torch.empty(50, dtype=torch.int32, device="cuda")
        d_sigma = torch.empty(50, dtype=torch.int64, device="cuda")
        d_spread = torch.empty(1, dtype=torch.int64, device="cuda")
        for p in (0.01, 0.05):
            im.im_select_seeds_async(g, ws, 50, 1024, p, 7, d_seeds, d_sigma)
            im.im_estimate_spread_async(g, ws, d_seeds, 50, 1024, p, 7, d_spread)
            im.im_workspace_status(ws)
            stream.synchronize()
            seeds, sigma = im.im_select_seeds(g, 50, 1024, p, 7)
            assert np.array_equal(d_seeds.cpu().numpy(), seeds)
            assert np.array_equal(d_sigma.cpu().numpy().astype(np.uint64), sigma)
            assert int(d_spread.item()) == int(sigma[-1])
    finally:
        im.im_set_stream(None)
        ws.close()


def test_invalid_inputs_keep_handles_usable(g2000):
    xadj, adj, g = g2000
    bad = [dict(K=-1), dict(K=2001), dict(R=0), dict(R=65537), dict(p=float("nan")),
           dict(p=-0.5), dict(p=1.5)]
    for b in bad:
        kw = dict(K=5, R=16, p=0.1)
        kw.update(b)
        with pytest.raises(im.IMError) as e:
            im.im_select_seeds(g, kw["K"], kw["R"], kw["p"], 1)
        assert e.value.code == im.IM_EINVAL
    with pytest.raises(im.IMError):
        im.im_estimate_spread(g, [0, 2000], 16, 0.1, 1)
    # n * R >= 2^32
    big = _graph(np.zeros(70001, dtype=np.int32), np.array([], dtype=np.int32))
    with pytest.raises(im.IMError) as e:
        im.im_select_seeds(big, 1, 65536, 0.1, 1)
    assert e.value.code == im.IM_EINVAL
    # asymmetric CSR and out-of-range ids
    with pytest.raises(im.IMError) as e:
        im.im_graph_create(np.array([0, 1, 1, 2], dtype=np.int32), np.array([1, 1], dtype=np.int32))
    assert e.value.code == im.IM_EINVAL
    with pytest.raises(im.IMError) as e:
        im.im_graph_create(np.array([0, 1, 2], dtype=np.int32), np.array([1, 5], dtype=np.int32))
    assert e.value.code == im.IM_EINVAL
    with pytest.raises(im.IMError) as e:
        im.im_graph_create(np.array([0, 2, 1, 2], dtype=np.int32), np.array([1, 2], dtype=np.int32))
    assert e.value.code == im.IM_EINVAL
    seeds, sigma = im.im_select_seeds(g, 10, 256, 0.01, 7)
    oseeds, osigma = oracle.select_seeds(xadj, adj, 10, 256, 0.01, 7)
    assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)


def test_concurrent_queries_on_streams_match_serial():
    """Independent queries on three streams with three workspaces overlap on
    the device; each result equals the same query run alone."""
    import torch

    xadj, adj = synth.workload_graph("powerlaw_n2000")
    g = _graph(xadj, adj)
    R, K, seed = 256, 10, 7
    ps = (0.005, 0.01, 0.05)
    alone = [im.im_select_seeds(g, K, R, p, seed) for p in ps]
    dev = torch.device("cuda", 0)
    streams = [torch.cuda.Stream(device=dev) for _ in ps]
    wss = [im.im_workspace_create(g, R) for _ in ps]
    d_seeds = torch.zeros((len(ps), K), dtype=torch.int32, device=dev)
    d_sigma = torch.zeros((len(ps), K), dtype=torch.int64, device=dev)
    d_spread = torch.zeros(len(ps), dtype=torch.int64, device=dev)
    for _ in range(2):
        for i, p in enumerate(ps):
            im.im_set_stream(streams[i])
            im.im_select_seeds_async(g, wss[i], K, R, p, seed, d_seeds[i], d_sigma[i])
            im.im_estimate_spread_async(g, wss[i], d_seeds[i], K, R, p, seed, d_spread[i:i + 1])
        torch.cuda.synchronize()
        for i, p in enumerate(ps):
            im.im_set_stream(streams[i])
            im.im_workspace_status(wss[i])
            assert np.array_equal(d_seeds[i].cpu().numpy(), alone[i][0])
            assert np.array_equal(d_sigma[i].cpu().numpy().astype(np.uint64), alone[i][1])
            assert int(d_spread[i].item()) == int(alone[i][1][-1])
    im.im_set_stream(None)
    for w_ in wss:
        w_.close()


@pytest.mark.parametrize("R", [20480, 20481, 32768])
def test_large_R_pool_in_global_memory_and_wide_spread_rows(R):
    """R above 20480 moves the lazy greedy's pool to global memory (20480 is
    the last R whose pool of one candidate fits the shared-memory budget), and
    R above 2048 gives spread rows wider than the register copy."""
    xadj, adj = synth.random_graph(300, 900, 6)
    g = _graph(xadj, adj)
    seeds, sigma = im.im_select_seeds(g, 5, R, 0.05, 7)
    oseeds, osigma = oracle.select_seeds(xadj, adj, 5, R, 0.05, 7)
    assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)
    assert im.im_estimate_spread(g, seeds, R, 0.05, 7) == int(osigma[-1])
    S = np.array([3, 77, 150, 3], dtype=np.int32)
    assert im.im_estimate_spread(g, S, R, 0.05, 7) == oracle.estimate_spread(xadj, adj, S, R, 0.05, 7)


@pytest.mark.parametrize("p", [0.02, 0.2])
def test_lane_ranges_on_gpu_sum_to_the_full_selection(p):
    """Two lane ranges computed one after the other on the GPU give the
    matching columns of the full tables, and summing the two ranges' marginal
    gains on the host before each commit (gain desc, id asc) reproduces the
    seeds and sigma*R that the GPU selects over the full range."""
    xadj, adj = synth.chung_lu(400, 1600, 2.3, 23)
    R, seed, K = 96, 7, 8
    g = _graph(xadj, adj)
    full_lab = im.im_debug_labels(g, R, p, seed)
    full_siz = im.im_debug_sizes(g, R, p, seed)
    shards = [np.arange(0, 40), np.arange(40, R)]
    tabs = [im.im_debug_tables_lanes(g, R, p, seed, lanes) for lanes in shards]
    for lanes, (lab, siz) in zip(shards, tabs):
        assert np.array_equal(lab, full_lab[:, lanes])
        assert np.array_equal(siz, full_siz[:, lanes])
    seeds, sigma = im.im_select_seeds(g, K, R, p, seed)
    S, total = [], 0
    for k in range(K):
        gsum = sum(oracle.marginal_gains(lab, siz, S).astype(np.int64) for lab, siz in tabs)
        gsum[S] = -1
        best = int(np.argmax(gsum))
        total += int(gsum[best])
        assert seeds[k] == best and int(sigma[k]) == total
        S.append(best)
