"""Sampling options and the FusedSampling variant on the GPU, bit-exact
against the oracle:

- per-edge probabilities w(u,v) (the paper's weight settings U[0, 0.1] and
  N(0.05, 0.025), Section 4): labels, sizes, seeds, sigma*R and spreads;
  unsorted neighbour lists (sorted with their weights at graph creation);
- the mixed hash (fmix32 of X_r XOR h): the same, every lane a candidate;
- IM_ALGO_FUSED_SAMPLING (one simulation at a time, no memo, CELF by RandCas
  on the fixed samples): the same seeds and sigma*R as the oracle and as the
  default path.
"""
import numpy as np
import pytest

import oracle
import paper_2008_03095_gb300 as im
from paper_2008_03095_gb300 import build as im_build
from paper_2008_03095_gb300 import synth

pytestmark = pytest.mark.gpu

W, MIX, FS = im.IM_SAMPLE_EDGE_WEIGHTS, im.IM_SAMPLE_MIXED_HASH, im.IM_ALGO_FUSED_SAMPLING


@pytest.fixture(scope="module", autouse=True)
def _lib():
    im_build.build()
    im.lib()


def _kw(flags, w):
    return dict(weights=w if flags & W else None, mix=bool(flags & MIX))


GRAPHS = [
    ("chung_lu_1200_hub", lambda: synth.chung_lu(1200, 6000, 2.1, 9)),
    ("random_300", lambda: synth.random_graph(300, 900, 6)),
]


@pytest.mark.parametrize("name,mk", GRAPHS)
@pytest.mark.parametrize("kind", ["uniform", "normal"])
@pytest.mark.parametrize("flags", [W, MIX, W | MIX])
@pytest.mark.parametrize("R", [1, 33, 256])
def test_tables_and_selection_with_options(name, mk, kind, flags, R):
    xadj, adj = mk()
    w = synth.edge_weights(xadj, adj, kind, 5)
    p = 0.05
    g = im.im_graph_create_weighted(xadj, adj, w)
    lab, siz = oracle.labels_ex(xadj, adj, R, p, 7, **_kw(flags, w))
    glab, gsiz = im.im_debug_tables_ex(g, R, p, 7, flags)
    assert np.array_equal(glab, lab)
    assert np.array_equal(gsiz, siz)
    K = 12
    oseeds, osigma = oracle.select_seeds_ex(xadj, adj, K, R, p, 7, **_kw(flags, w))
    seeds, sigma = im.im_select_seeds_ex(g, K, R, p, 7, flags)
    assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)
    S = np.array([0, 5, 5, 77], dtype=np.int32)
    assert im.im_estimate_spread_ex(g, S, R, p, 7, flags) == oracle.estimate_spread_ex(
        xadj, adj, S, R, p, 7, **_kw(flags, w))
    g.close()


def test_weights_extremes_and_uniform_equivalence():
    xadj, adj = synth.chung_lu(900, 4000, 2.3, 12)
    n = 900
    src = np.repeat(np.arange(n), np.diff(xadj))
    sel = ((np.minimum(src, adj) * 7 + np.maximum(src, adj) * 13) % 3) == 0
    w01 = sel.astype(np.float64)  # certain edges and impossible ones
    g = im.im_graph_create_weighted(xadj, adj, w01)
    lab, siz = oracle.labels_ex(xadj, adj, 40, 0.0, 3, weights=w01)
    assert np.array_equal(im.im_debug_tables_ex(g, 40, 0.0, 3, W)[0], lab)
    g.close()
    # every weight = p: the weighted path gives the uniform-p result
    wp = np.full(adj.shape[0], 0.05)
    g = im.im_graph_create_weighted(xadj, adj, wp)
    a = im.im_select_seeds(g, 10, 128, 0.05, 3)
    b = im.im_select_seeds_ex(g, 10, 128, 0.9, 3, W)  # p ignored with weights
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    g.close()


def test_unsorted_lists_keep_their_weights():
    xadj, adj = synth.chung_lu(700, 3000, 2.2, 13)
    w = synth.edge_weights(xadj, adj, "uniform", 6)
    rng = np.random.default_rng(0)
    adj2, w2 = adj.copy(), w.copy()
    for u in range(700):
        a, b = xadj[u], xadj[u + 1]
        perm = rng.permutation(b - a)
        adj2[a:b] = adj[a:b][perm]
        w2[a:b] = w[a:b][perm]
    g = im.im_graph_create_weighted(xadj, adj2, w2)
    oseeds, osigma = oracle.select_seeds_ex(xadj, adj2, 10, 64, 0.0, 9, weights=w2)
    seeds, sigma = im.im_select_seeds_ex(g, 10, 64, 0.0, 9, W)
    assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)
    g.close()


@pytest.mark.parametrize("kind", ["uniform", "normal"])
def test_weighted_netphy_shape_full_parity(kind):
    """The NetHEP-shaped workload (n = 15,233, R = 1024, K = 50) with the
    paper's two weight settings, through the async API as bench.py calls it."""
    import torch

    xadj, adj = synth.workload_graph("powerlaw_n15233")
    w = synth.edge_weights(xadj, adj, kind, 15233)
    K, R = 50, 1024
    oracle.use_all_cores(True)
    try:
        oseeds, osigma = oracle.select_seeds_ex(xadj, adj, K, R, 0.0, 7, weights=w)
    finally:
        oracle.use_all_cores(False)
    g = im.im_graph_create_weighted(xadj, adj, w)
    ws = im.im_workspace_create(g, R)
    im.im_set_stream(torch.cuda.current_stream())
    d_seeds = torch.empty(K, dtype=torch.int32, device="cuda")
    d_sigma = torch.empty(K, dtype=torch.int64, device="cuda")
    d_spread = torch.empty(1, dtype=torch.int64, device="cuda")
    im.im_select_seeds_ex_async(g, ws, K, R, 0.0, 7, W, d_seeds, d_sigma)
    im.im_estimate_spread_ex_async(g, ws, d_seeds, K, R, 0.0, 7, W, d_spread)
    im.im_workspace_status(ws)
    im.im_set_stream(None)
    assert np.array_equal(d_seeds.cpu().numpy(), oseeds)
    assert np.array_equal(d_sigma.cpu().numpy().astype(np.uint64), osigma)
    assert int(d_spread.cpu().numpy()[0]) == int(osigma[-1])
    ws.close()
    g.close()


@pytest.mark.parametrize("flags", [0, W, MIX])
@pytest.mark.parametrize("R,p", [(1, 0.3), (48, 0.05), (64, 0.0), (32, 1.0)])
def test_fused_sampling_variant_matches_oracle_and_default_path(flags, R, p):
    xadj, adj = synth.chung_lu(600, 2400, 2.3, 14)
    w = synth.edge_weights(xadj, adj, "uniform", 7)
    g = im.im_graph_create_weighted(xadj, adj, w)
    K = 8
    oseeds, osigma = oracle.select_seeds_ex(xadj, adj, K, R, p, 11, **_kw(flags, w))
    fseeds, fsigma = im.im_select_seeds_ex(g, K, R, p, 11, flags | FS)
    assert np.array_equal(fseeds, oseeds) and np.array_equal(fsigma, osigma)
    dseeds, dsigma = im.im_select_seeds_ex(g, K, R, p, 11, flags)
    assert np.array_equal(dseeds, fseeds) and np.array_equal(dsigma, fsigma)
    g.close()


def test_option_errors():
    xadj, adj = synth.random_graph(100, 300, 3)
    g = im.im_graph_create(xadj, adj)
    for call in (lambda: im.im_select_seeds_ex(g, 3, 8, 0.1, 1, W),
                 lambda: im.im_select_seeds_ex(g, 3, 8, 0.1, 1, 64),
                 lambda: im.im_estimate_spread_ex(g, [1], 8, 0.1, 1, W)):
        with pytest.raises(im.IMError) as e:
            call()
        assert e.value.code == im.IM_EINVAL
    ws = im.im_workspace_create(g, 8)
    import torch
    d = torch.empty(3, dtype=torch.int32, device="cuda")
    s = torch.empty(3, dtype=torch.int64, device="cuda")
    with pytest.raises(im.IMError) as e:
        im.im_select_seeds_ex_async(g, ws, 3, 8, 0.1, 1, FS, d, s)
    assert e.value.code == im.IM_EINVAL
    ws.close()
    g.close()
    w = np.full(adj.shape[0], 0.2)
    w[0] = 0.3  # the reverse arc keeps 0.2
    with pytest.raises(im.IMError) as e:
        im.im_graph_create_weighted(xadj, adj, w)
    assert e.value.code == im.IM_EINVAL
    w = np.full(adj.shape[0], 1.5)
    with pytest.raises(im.IMError) as e:
        im.im_graph_create_weighted(xadj, adj, w)
    assert e.value.code == im.IM_EINVAL
