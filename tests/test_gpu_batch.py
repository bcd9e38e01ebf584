"""Batched persistent launch (many uneven queries in one kernel launch): every
query's seeds and sigma*R equal the oracle's on its own and the single-query
GPU path's, on repeated runs, after autotuning, under CUDA-graph capture, and
with a device budget run out."""
import numpy as np
import pytest

import oracle
import paper_2008_03095_gb300 as im
from paper_2008_03095_gb300 import build as im_build
from paper_2008_03095_gb300 import synth

pytestmark = pytest.mark.gpu

W, MIX = im.IM_SAMPLE_EDGE_WEIGHTS, im.IM_SAMPLE_MIXED_HASH


@pytest.fixture(scope="module", autouse=True)
def _lib():
    im_build.build()
    im.lib()
    yield
    im.im_debug_clear_overrides()


@pytest.fixture(scope="module")
def small_batch():
    """24 uneven queries over 12 graphs (sizes 120..6000 vertices, R from 1
    to 512, p from 0 to 1, weighted and mixed sampling among them), with the
    oracle's answer for each."""
    rng = np.random.default_rng(2024)
    graphs, specs = [], []
    for gi in range(12):
        n = int(rng.choice([120, 300, 800, 2000, 6000]))
        if gi % 3 == 0:
            xadj, adj = synth.random_graph(n, 3 * n, 100 + gi)
        else:
            xadj, adj = synth.chung_lu(n, int(n * rng.uniform(2, 8)), rng.uniform(2.0, 3.0), 100 + gi)
        w = synth.edge_weights(xadj, adj, "uniform" if gi % 2 else "normal", gi)
        graphs.append((xadj, adj, w))
    queries, expected = [], []
    for qi in range(24):
        gi = qi % 12
        xadj, adj, w = graphs[gi]
        n = xadj.shape[0] - 1
        R = int(rng.choice([1, 33, 64, 256, 512]))
        p = float(rng.choice([0.0, 0.003, 0.02, 0.1, 0.4, 1.0]))
        flags = int(rng.choice([0, 0, 0, W, MIX, W | MIX]))
        K = int(min(rng.integers(1, 40), n))
        q = dict(graph=gi, K=K, R=R, p=p, rng_seed=int(rng.integers(0, 2 ** 32)), flags=flags)
        queries.append(q)
        expected.append(oracle.select_seeds_ex(
            xadj, adj, K, R, p, q["rng_seed"], weights=w if flags & W else None,
            mix=bool(flags & MIX)))
    handles = [im.im_graph_create_weighted(x, a, w) for x, a, w in graphs]
    yield handles, queries, expected
    for g in handles:
        g.close()


def _check(b, expected):
    seeds, sigma, status = im.im_batch_results(b)
    assert np.all(status == 0)
    for i, (es, eg) in enumerate(expected):
        assert np.array_equal(seeds[i], es), (i, seeds[i], es)
        assert np.array_equal(sigma[i], eg), (i, sigma[i], eg)


def test_batch_matches_oracle_per_query(small_batch):
    handles, queries, expected = small_batch
    b = im.im_batch_create(handles, queries)
    info = im.im_batch_info(b)
    assert info["queries"] == 24 and info["items"] >= 24 * 3
    im.im_batch_run_async(b)
    _check(b, expected)
    im.im_batch_run_async(b)  # a second run over the same arena
    _check(b, expected)
    b.close()


def test_batch_matches_single_query_path(small_batch):
    handles, queries, _ = small_batch
    b = im.im_batch_create(handles, queries)
    im.im_batch_run_async(b)
    seeds, sigma, _ = im.im_batch_results(b)
    for i, q in enumerate(queries):
        s1, g1 = im.im_select_seeds_ex(handles[q["graph"]], q["K"], q["R"], q["p"], q["rng_seed"],
                                       q["flags"])
        assert np.array_equal(seeds[i], s1) and np.array_equal(sigma[i], g1)
    b.close()


def test_autotune_keeps_results_and_cache_roundtrip(small_batch, tmp_path):
    handles, queries, expected = small_batch
    im.im_autotune_cache_clear()
    b = im.im_batch_create(handles, queries)
    before = im.im_batch_info(b)["levels"]
    im.im_batch_autotune(b, 2)
    im.im_batch_run_async(b)
    _check(b, expected)
    path = str(tmp_path / "tune.txt")
    im.im_autotune_cache_save(path)
    lines = [l for l in open(path) if not l.startswith("#")]
    assert len(lines) >= 1
    im.im_autotune_cache_clear()
    im.im_autotune_cache_load(path)
    b2 = im.im_batch_create(handles, queries)  # planned from the loaded cache
    assert im.im_batch_info(b2)["levels"] == im.im_batch_info(b)["levels"]
    im.im_batch_run_async(b2)
    _check(b2, expected)
    b.close()
    b2.close()
    del before


def test_batch_run_captured_in_a_cuda_graph(small_batch):
    import torch

    handles, queries, expected = small_batch
    b = im.im_batch_create(handles, queries)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        im.im_set_stream(s)
        with torch.cuda.graph(graph, stream=s):
            im.im_batch_run_async(b)
    im.im_set_stream(None)
    torch.cuda.synchronize()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        _check(b, expected)
    b.close()


def test_uneven_instances_of_the_batched_recipe_match_single_queries():
    """48 instances of the uneven recipe (n log-uniform in [500, 20000],
    m/n in [2, 15], exponent in [2, 3], p log-uniform in [0.001, 0.1],
    R in {256, 1024, 2048}, K in [5, 100])."""
    inst = synth.batched_instances(count=48, seed=41, n_range=(500, 20000))
    handles = [im.im_graph_create(*synth.instance_graph(x)) for x in inst]
    queries = [dict(graph=i, K=x["K"], R=x["R"], p=x["p"], rng_seed=x["rng_seed"])
               for i, x in enumerate(inst)]
    b = im.im_batch_create(handles, queries)
    im.im_batch_run_async(b)
    seeds, sigma, status = im.im_batch_results(b)
    assert np.all(status == 0)
    for i, q in enumerate(queries):
        s1, g1 = im.im_select_seeds(handles[i], q["K"], q["R"], q["p"], q["rng_seed"])
        assert np.array_equal(seeds[i], s1) and np.array_equal(sigma[i], g1), i
    # the smallest few against the oracle directly
    order = sorted(range(len(inst)), key=lambda i: inst[i]["n"] * inst[i]["R"])[:3]
    for i in order:
        xadj, adj = synth.instance_graph(inst[i])
        es, eg = oracle.select_seeds(xadj, adj, inst[i]["K"], inst[i]["R"], inst[i]["p"],
                                     inst[i]["rng_seed"])
        assert np.array_equal(seeds[i], es) and np.array_equal(sigma[i], eg)
    b.close()
    for g in handles:
        g.close()


def test_round_budget_run_out_in_a_batch(small_batch):
    handles, queries, expected = small_batch
    im.im_debug_override(im.IM_OVR_CELF_ROUND_CAP, 1)
    try:
        b = im.im_batch_create(handles, queries)  # the budget is taken at creation
    finally:
        im.im_debug_override(im.IM_OVR_CELF_ROUND_CAP, 0)
    im.im_batch_run_async(b)
    with pytest.raises(im.IMError) as e:
        im.im_batch_results(b)
    assert e.value.code == im.IM_ETIMEOUT
    _, _, status = im.im_batch_results(b, check=False)
    assert np.any(status == im.IM_ETIMEOUT)
    assert set(np.unique(status).tolist()) <= {0, im.IM_ETIMEOUT}
    b.close()
    b = im.im_batch_create(handles, queries)
    im.im_batch_run_async(b)
    _check(b, expected)
    b.close()


def test_batch_argument_errors(small_batch):
    handles, queries, _ = small_batch
    bad = [dict(queries[0], graph=99), dict(queries[0], R=20000), dict(queries[0], K=0),
           dict(queries[0], flags=im.IM_ALGO_FUSED_SAMPLING), dict(queries[0], p=1.5)]
    for q in bad:
        with pytest.raises(im.IMError) as e:
            im.im_batch_create(handles, [q])
        assert e.value.code == im.IM_EINVAL
