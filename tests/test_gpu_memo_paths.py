"""The size memo's walks (Section 3.3): a one-block-per-lane probe of the
union-find table picks per-warp root-count accumulators where a sample holds
a large component (walking only a warp's listed non-root slots when those are
few), and the path-compressing walk otherwise. All give the oracle's tables
and seeds; the work counters say which one ran.
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
    oracle.use_all_cores()


@pytest.fixture(scope="module")
def c2():
    xadj, adj = synth.workload_graph("powerlaw_n15233")
    g = im.im_graph_create(xadj, adj)
    yield xadj, adj, g
    g.close()


def _select_with_stats(g, K, R, p, seed):
    torch = pytest.importorskip("torch")
    ws = im.im_workspace_create(g, R)
    im.im_set_stream(torch.cuda.current_stream())
    try:
        d_seeds = torch.empty(K, dtype=torch.int32, device="cuda")
        d_sigma = torch.empty(K, dtype=torch.int64, device="cuda")
        im.im_workspace_stats(ws)
        im.im_select_seeds_async(g, ws, K, R, p, seed, d_seeds, d_sigma)
        im.im_workspace_status(ws)
        st = im.im_workspace_stats(ws)
        return d_seeds.cpu().numpy(), d_sigma.cpu().numpy().astype(np.uint64), st
    finally:
        im.im_set_stream(None)
        ws.close()


@pytest.mark.parametrize("p,accumulate", [(0.05, 1), (0.01, 0)])
def test_both_walks_equal_oracle(c2, p, accumulate):
    """On the 15k-vertex power-law graph a sample's largest component holds
    about 9% of the vertices at p = 0.05 and 0.1% at p = 0.01."""
    xadj, adj, g = c2
    R, K = 1024, 30
    seeds, sigma, st = _select_with_stats(g, K, R, p, 7)
    assert st["memo_accumulators"] == accumulate
    assert st["memo_live"] == 0  # a quarter of the slots are not roots at p = 0.05
    lab, siz = oracle.labels(xadj, adj, R, p, 7)
    assert np.array_equal(im.im_debug_labels(g, R, p, 7), lab)
    assert np.array_equal(im.im_debug_sizes(g, R, p, 7), siz)
    want_seeds, want_sigma = oracle.greedy_from_tables(lab, siz, K)
    assert np.array_equal(seeds, want_seeds) and np.array_equal(sigma, want_sigma)


def test_giant_component_graph_takes_accumulators():
    xadj, adj = synth.chung_lu(200_000, 1_000_000, 2.2, 77)
    g = im.im_graph_create(xadj, adj)
    try:
        R = 64
        seeds, sigma, st = _select_with_stats(g, 10, R, 0.05, 3)
        assert st["memo_accumulators"] == 1 and st["memo_live"] == 0
        lanes = np.array([0, 17, 63], dtype=np.int32)
        lab, siz = oracle.labels_lanes(xadj, adj, R, 0.05, 3, lanes)
        glab, gsiz = im.im_debug_tables_lanes(g, R, 0.05, 3, lanes)
        assert np.array_equal(glab, lab) and np.array_equal(gsiz, siz)
    finally:
        g.close()


def test_few_non_roots_take_the_listed_walk():
    """A 1M-vertex power-law graph at p = 0.01: its largest component holds
    about 5% of the vertices, and about 10% of the slots are not roots."""
    xadj, adj = synth.chung_lu(1_000_000, 8_750_000, 2.2, 42)
    g = im.im_graph_create(xadj, adj)
    try:
        R, p = 64, 0.01
        seeds, sigma, st = _select_with_stats(g, 10, R, p, 5)
        assert st["memo_accumulators"] == 1 and st["memo_live"] == 1
        lanes = np.array([0, 31, 63], dtype=np.int32)
        lab, siz = oracle.labels_lanes(xadj, adj, R, p, 5, lanes)
        glab, gsiz = im.im_debug_tables_lanes(g, R, p, 5, lanes)
        assert np.array_equal(glab, lab) and np.array_equal(gsiz, siz)
        assert im.im_estimate_spread(g, seeds, R, p, 5) == int(sigma[-1])
    finally:
        g.close()
