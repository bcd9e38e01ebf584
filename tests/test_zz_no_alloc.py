"""im_estimate_spread_noalloc: the spread estimate computed in the library's
static device scratch, checked against im_estimate_spread (which computes the
same quantity in allocated workspaces) and the oracle. Collected last so that
it also runs after every other GPU test in the same process."""
import numpy as np
import pytest

import oracle
import paper_2008_03095_gb300 as im
from paper_2008_03095_gb300 import build as im_build
from paper_2008_03095_gb300 import synth

pytestmark = pytest.mark.gpu

LIM = im.NOALLOC_LIMITS


@pytest.fixture(scope="module", autouse=True)
def _lib():
    im_build.build()
    im.lib()


def _graph(xadj, adj):
    return im.im_graph_create(xadj, adj)


@pytest.mark.parametrize("R,p", [(256, 0.01), (33, 0.1), (1, 0.3), (LIM["IM_NOALLOC_MAX_R"], 1.0)])
def test_two_calls_in_a_row_match_allocating_path(R, p):
    xadj, adj = synth.chung_lu(2000, 8000, 2.5, 1)
    g = _graph(xadj, adj)
    rng = np.random.default_rng(R)
    S1 = rng.integers(0, 2000, size=10)
    S2 = rng.integers(0, 2000, size=3)
    S2 = np.concatenate([S2, S2[:1]])  # a duplicate seed counts once
    # two calls in a row on the static scratch, then the allocating path
    a1 = im.im_estimate_spread_noalloc(g, S1, R, p, 7)
    a2 = im.im_estimate_spread_noalloc(g, S2, R, p, 7)
    assert a1 == im.im_estimate_spread(g, S1, R, p, 7)
    assert a2 == im.im_estimate_spread(g, S2, R, p, 7)
    # and again after the allocating path ran (nothing stale in the scratch)
    assert im.im_estimate_spread_noalloc(g, S1, R, p, 7) == a1


def test_matches_oracle_and_edge_cases():
    xadj, adj = synth.chung_lu(1200, 6000, 2.1, 9)
    g = _graph(xadj, adj)
    S = np.array([3, 17, 17, 900], dtype=np.int32)
    assert im.im_estimate_spread_noalloc(g, S, 64, 0.05, 11) == oracle.estimate_spread(
        xadj, adj, S, 64, 0.05, 11)
    assert im.im_estimate_spread_noalloc(g, [], 64, 0.05, 11) == 0
    assert im.im_estimate_spread_noalloc(g, [5], 64, 0.0, 11) == 64  # p = 0: only the seed


def test_limits_are_rejected_before_device_work():
    xadj, adj = synth.chung_lu(2000, 8000, 2.5, 1)
    g = _graph(xadj, adj)
    with pytest.raises(im.IMError) as e:
        im.im_estimate_spread_noalloc(g, [1], LIM["IM_NOALLOC_MAX_R"] + 1, 0.1, 7)
    assert e.value.code == im.IM_EINVAL
    with pytest.raises(im.IMError) as e:
        im.im_estimate_spread_noalloc(g, [2000], 8, 0.1, 7)  # id out of range
    assert e.value.code == im.IM_EINVAL
    big = LIM["IM_NOALLOC_MAX_N"] + 1
    xb, ab = synth.random_graph(big, big, 3)
    gb = _graph(xb, ab)
    with pytest.raises(im.IMError) as e:
        im.im_estimate_spread_noalloc(gb, [0], 8, 0.1, 7)
    assert e.value.code == im.IM_EINVAL
    # the library stays usable afterwards
    assert im.im_estimate_spread_noalloc(g, [1], 8, 0.1, 7) == im.im_estimate_spread(g, [1], 8, 0.1, 7)


def test_calls_leave_free_device_memory_unchanged():
    """The property the entry point exists for: once the static region is in
    place (first call), further calls take no device memory at all."""
    import torch

    xadj, adj = synth.chung_lu(2000, 8000, 2.5, 1)
    g = _graph(xadj, adj)
    S = np.array([1, 2, 3, 500], dtype=np.int32)
    want = im.im_estimate_spread(g, S, 128, 0.05, 7)  # the allocating path, first
    assert im.im_estimate_spread_noalloc(g, S, 128, 0.05, 7) == want  # warm-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for R in (1, 64, 128, LIM["IM_NOALLOC_MAX_R"]):
        im.im_estimate_spread_noalloc(g, S, R, 0.05, 7)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    g.close()


def test_succeeds_while_another_allocator_holds_the_free_memory():
    """A caching allocator that has taken almost all free device memory leaves
    the allocating entry point nothing to work with, but not this one."""
    import torch

    xadj, adj = synth.chung_lu(2000, 8000, 2.5, 1)
    g = _graph(xadj, adj)
    S = np.array([7, 8, 9], dtype=np.int32)
    want = im.im_estimate_spread(g, S, 256, 0.02, 7)
    assert im.im_estimate_spread_noalloc(g, S, 256, 0.02, 7) == want
    torch.cuda.synchronize()
    hog = None
    try:
        free = torch.cuda.mem_get_info()[0]
        # leave 256 MiB for the driver (kernel launches, local memory)
        hog = torch.empty(max(free - (256 << 20), 0), dtype=torch.uint8, device="cuda")
        g2 = None
        for _ in range(3):
            assert im.im_estimate_spread_noalloc(g, S, 256, 0.02, 7) == want
        # a fresh graph's allocating query needs a workspace larger than what is left
        xb, ab = synth.chung_lu(30000, 200000, 2.3, 5)
        g2 = _graph(xb, ab) if torch.cuda.mem_get_info()[0] > (64 << 20) else None
        if g2 is not None:
            with pytest.raises(im.IMError) as e:
                im.im_estimate_spread(g2, [0], 65536, 0.02, 7)  # n*R*4 = 7.9 GB of workspace
            assert e.value.code == im.IM_ENOMEM
            g2.close()
    finally:
        del hog
        torch.cuda.empty_cache()
    g.close()
