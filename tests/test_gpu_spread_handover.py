"""The spread's hand-over from the multi-source BFS to the samples' components
(Algorithm 4 on the fixed samples of Eq. 2; the library switches on tables
larger than L2 once a BFS frontier passes n/16 vertices, then marks the
seeds' roots and counts the slots under a marked root): sigma*R equal to
the oracle's per-sample BFS with and without the hand-over, under the
sampling options, with duplicate and empty seed sets, and equal to the lazy
greedy's sigma*R of its own seeds.
"""
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


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


def _l2_bytes(torch):
    return int(torch.cuda.get_device_properties(0).L2_cache_size)


def _spread(torch, g, seeds, R, p, seed, flags=0):
    """sigma*R through the async entry point, and the query's work counters."""
    ws = im.im_workspace_create(g, R)
    stream = torch.cuda.current_stream()
    im.im_set_stream(stream)
    try:
        d_seeds = torch.from_numpy(np.ascontiguousarray(seeds, dtype=np.int32)).cuda()
        d_sigma = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        im.im_workspace_stats(ws)
        im.im_estimate_spread_ex_async(g, ws, d_seeds, len(seeds), R, p, seed, flags, d_sigma)
        im.im_workspace_status(ws)
        stats = im.im_workspace_stats(ws)
        return int(d_sigma.item()), stats
    finally:
        im.im_set_stream(None)
        ws.close()


def _top_degree(xadj, k):
    return np.argsort(-np.diff(xadj), kind="stable")[:k].astype(np.int32)


@pytest.fixture(scope="module")
def giant():
    """A power-law graph whose 256-lane table (200 MB) exceeds L2 and whose
    samples at p = 0.05 hold a giant component."""
    xadj, adj = synth.chung_lu(200_000, 1_000_000, 2.2, 77)
    g = im.im_graph_create(xadj, adj)
    yield xadj, adj, g
    g.close()


def test_handover_equals_oracle(torch, giant):
    xadj, adj, g = giant
    R, p = 256, 0.05
    assert (len(xadj) - 1) * R * 4 > _l2_bytes(torch)
    seeds = _top_degree(xadj, 20)
    got, st = _spread(torch, g, seeds, R, p, 7)
    assert st["spread_components"] == 1
    assert got == oracle.estimate_spread(xadj, adj, seeds, R, p, 7)
    # the blocking call takes the same path
    assert im.im_estimate_spread(g, seeds, R, p, 7) == got


def test_handover_lane_count_not_a_multiple_of_four(torch, giant):
    """The count after the hand-over reads a table row lane by lane when R is
    not a multiple of 4 (rows are not 16-byte aligned)."""
    xadj, adj, g = giant
    R, p = 250, 0.05
    assert (len(xadj) - 1) * R * 4 > _l2_bytes(torch)
    seeds = _top_degree(xadj, 12)
    got, st = _spread(torch, g, seeds, R, p, 13)
    assert st["spread_components"] == 1
    assert got == oracle.estimate_spread(xadj, adj, seeds, R, p, 13)


@pytest.mark.parametrize("flags", [W, MIX, W | MIX])
def test_handover_sampling_options_equal_oracle(torch, flags):
    xadj, adj = synth.chung_lu(200_000, 1_000_000, 2.2, 77)
    w = synth.edge_weights(xadj, adj, "uniform", 3)
    g = im.im_graph_create_weighted(xadj, adj, w)
    try:
        R, p = 256, 0.05
        seeds = _top_degree(xadj, 10)
        got, st = _spread(torch, g, seeds, R, p, 11, flags)
        assert st["spread_components"] == 1
        want = oracle.estimate_spread_ex(xadj, adj, seeds, R, p, 11,
                                         weights=w if flags & W else None, mix=bool(flags & MIX))
        assert got == want
    finally:
        g.close()


def test_handover_duplicate_and_empty_seed_sets(torch, giant):
    xadj, adj, g = giant
    R, p = 256, 0.05
    seeds = _top_degree(xadj, 8)
    once, _ = _spread(torch, g, seeds, R, p, 5)
    twice, st = _spread(torch, g, np.concatenate([seeds, seeds[::-1], seeds[:3]]), R, p, 5)
    assert st["spread_components"] == 1 and twice == once
    none, st = _spread(torch, g, np.zeros(0, dtype=np.int32), R, p, 5)
    assert none == 0 and st["spread_components"] == 0


def test_spread_of_selected_seeds_equals_lazy_greedy_sigma(torch, giant):
    xadj, adj, g = giant
    R, p = 256, 0.05
    seeds, sigma = im.im_select_seeds(g, 25, R, p, 9)
    got, st = _spread(torch, g, seeds, R, p, 9)
    assert st["spread_components"] == 1
    assert got == int(sigma[-1])
    for k in (1, 5):  # prefixes: the hand-over happens or not, the value is the same
        assert _spread(torch, g, seeds[:k], R, p, 9)[0] == int(sigma[k - 1])


def test_small_reach_keeps_the_bfs(torch):
    """A low-skew clustered graph at p = 0.01: the table exceeds L2 but the
    samples hold only small components, so the BFS finishes by itself."""
    xadj, adj = synth.workload_graph("clustered_n334863")
    g = im.im_graph_create(xadj, adj)
    try:
        R, p = 128, 0.01
        assert (len(xadj) - 1) * R * 4 > _l2_bytes(torch)
        seeds = _top_degree(xadj, 50)
        got, st = _spread(torch, g, seeds, R, p, 7)
        assert st["spread_components"] == 0
        assert got == oracle.estimate_spread(xadj, adj, seeds, R, p, 7)
    finally:
        g.close()
