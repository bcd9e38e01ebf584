"""Failure paths on the GPU, made to happen without faulting anything: device
loop budgets are shrunk through the test-only override so that a healthy
query runs out of them (IM_ETIMEOUT), and a device allocation is made to fail
on the host (IM_ENOMEM). After each failure the same handles answer a normal
query with the oracle's result."""
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


@pytest.fixture(autouse=True)
def clear_overrides():
    im.im_debug_clear_overrides()
    yield
    im.im_debug_clear_overrides()


def _code(fn, *args):
    with pytest.raises(im.IMError) as e:
        fn(*args)
    return e.value.code


@pytest.fixture(scope="module")
def small():
    xadj, adj = synth.chung_lu(2000, 8000, 2.5, 1)
    K, R, p = 10, 256, 0.01
    oseeds, osigma = oracle.select_seeds(xadj, adj, K, R, p, 7)
    return xadj, adj, K, R, p, oseeds, osigma


def _check_normal_query(g, small):
    xadj, adj, K, R, p, oseeds, osigma = small
    seeds, sigma = im.im_select_seeds(g, K, R, p, 7)
    assert np.array_equal(seeds, oseeds) and np.array_equal(sigma, osigma)
    assert im.im_estimate_spread(g, seeds, R, p, 7) == int(osigma[-1])


def test_celf_round_budget_runs_out(small):
    import torch

    xadj, adj = synth.chung_lu(2000, 8000, 2.5, 1)
    g = im.im_graph_create(xadj, adj)
    K, R, p = 100, 256, 0.1  # a giant component: many rounds after the first commit
    ws = im.im_workspace_create(g, R)
    d_seeds = torch.empty(K, dtype=torch.int32, device="cuda")
    d_sigma = torch.empty(K, dtype=torch.int64, device="cuda")
    im.im_set_stream(torch.cuda.current_stream())
    im.im_workspace_stats(ws)
    im.im_select_seeds_async(g, ws, K, R, p, 7, d_seeds, d_sigma)
    im.im_workspace_status(ws)
    rounds = im.im_workspace_stats(ws)["celf_rounds"]
    assert rounds >= 2, rounds
    im.im_debug_override(im.IM_OVR_CELF_ROUND_CAP, 1)
    im.im_select_seeds_async(g, ws, K, R, p, 7, d_seeds, d_sigma)
    assert _code(im.im_workspace_status, ws) == im.IM_ETIMEOUT
    assert _code(im.im_select_seeds, g, K, R, p, 7) == im.IM_ETIMEOUT
    im.im_debug_override(im.IM_OVR_CELF_ROUND_CAP, 0)
    im.im_set_stream(None)
    ws.close()
    _check_normal_query(g, small)
    g.close()


def test_union_find_budget_runs_out(small):
    xadj, adj = small[0], small[1]
    g = im.im_graph_create(xadj, adj)
    im.im_debug_override(im.IM_OVR_UF_CAP, 1)
    # p = 1: one component per connected part, so walks longer than one step
    assert _code(im.im_debug_labels, g, 64, 1.0, 7) == im.IM_ETIMEOUT
    im.im_debug_override(im.IM_OVR_UF_CAP, 0)
    lab, _ = oracle.labels(xadj, adj, 64, 1.0, 7)
    assert np.array_equal(im.im_debug_labels(g, 64, 1.0, 7), lab)
    _check_normal_query(g, small)
    g.close()


def test_spread_level_budget_runs_out(small):
    xadj, adj = small[0], small[1]
    g = im.im_graph_create(xadj, adj)
    im.im_debug_override(im.IM_OVR_SPREAD_LEVEL_CAP, 1)
    assert _code(im.im_estimate_spread, g, [0, 1], 64, 1.0, 7) == im.IM_ETIMEOUT
    im.im_debug_override(im.IM_OVR_SPREAD_LEVEL_CAP, 0)
    assert im.im_estimate_spread(g, [0, 1], 64, 1.0, 7) == oracle.estimate_spread(
        xadj, adj, [0, 1], 64, 1.0, 7)
    _check_normal_query(g, small)
    g.close()


def test_allocation_failure_in_query_keeps_graph_usable(small):
    import torch

    xadj, adj = small[0], small[1]
    g = im.im_graph_create(xadj, adj)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # the query's internal workspace is the next allocation; fail its 1st,
    # then (a fresh attempt) its 7th buffer
    for k in (1, 7):
        im.im_debug_override(im.IM_OVR_FAIL_ALLOC, k)
        assert _code(im.im_select_seeds, g, 10, 256, 0.01, 7) == im.IM_ENOMEM
        im.im_debug_override(im.IM_OVR_FAIL_ALLOC, 0)
        # the partial workspace was released
        assert abs(torch.cuda.mem_get_info()[0] - free0) <= (8 << 20)
    _check_normal_query(g, small)
    g.close()


def test_allocation_failure_in_graph_create_and_workspace(small):
    xadj, adj = small[0], small[1]
    for k in (1, 2, 5):
        im.im_debug_override(im.IM_OVR_FAIL_ALLOC, k)
        assert _code(im.im_graph_create, xadj, adj) == im.IM_ENOMEM
    im.im_debug_override(im.IM_OVR_FAIL_ALLOC, 0)
    g = im.im_graph_create(xadj, adj)
    im.im_debug_override(im.IM_OVR_FAIL_ALLOC, 3)
    assert _code(im.im_workspace_create, g, 256) == im.IM_ENOMEM
    im.im_debug_override(im.IM_OVR_FAIL_ALLOC, 0)
    ws = im.im_workspace_create(g, 256)
    ws.close()
    _check_normal_query(g, small)
    g.close()

