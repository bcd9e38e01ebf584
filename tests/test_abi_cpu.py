"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function declared in include/im.h, and validates arguments before any
device call."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import paper_2008_03095_gb300 as im
from paper_2008_03095_gb300 import build as im_build


@pytest.fixture(scope="module")
def L():
    im_build.build()
    return im.lib()


def test_header_declares_the_boundary():
    names = set(im.header_functions())
    for need in ("im_graph_create", "im_graph_destroy", "im_select_seeds", "im_estimate_spread",
                 "im_last_error", "im_set_stream", "im_debug_labels", "im_debug_sizes",
                 "im_select_seeds_async", "im_estimate_spread_async", "im_workspace_create"):
        assert need in names


def test_library_exports_every_header_function(L):
    missing = []
    for name in im.header_functions():
        try:
            getattr(L, name)
        except AttributeError:
            missing.append(name)
    assert not missing, missing


def test_library_is_in_tree_and_loaded(L):
    path = im.library_path()
    assert path.endswith("libim_gb300.so")
    with open("/proc/self/maps") as f:
        assert path in f.read()


def test_sampling_threshold_matches_oracle(L):
    for p in (0.0, 1.0, 0.5, 0.01, 0.005, 0.05, 1e-9, 0.999999, 2.0 ** -32, 0.3):
        assert im.im_sampling_threshold(p) == oracle.threshold(p)
    for bad in (-0.1, 1.0000001, math.nan, math.inf):
        with pytest.raises(im.IMError) as e:
            im.im_sampling_threshold(bad)
        assert e.value.code == im.IM_EINVAL


def test_graph_create_rejects_bad_arguments_on_host(L):
    cases = [
        (np.array([0], dtype=np.int32), np.array([], dtype=np.int32)),         # n = 0
        (np.array([1, 2], dtype=np.int32), np.array([0, 0], dtype=np.int32)),  # xadj[0] != 0
        (np.array([0, 3], dtype=np.int32), np.array([0, 0], dtype=np.int32)),  # xadj[n] != 2m
    ]
    for xadj, adj in cases:
        with pytest.raises(im.IMError) as e:
            im.im_graph_create(xadj, adj)
        assert e.value.code == im.IM_EINVAL
        assert im.im_last_error()
    out = ctypes.c_void_p()
    assert L.im_graph_create(3, 0, None, None, ctypes.byref(out)) == im.IM_EINVAL


def test_queries_reject_null_handles(L):
    assert L.im_select_seeds(None, 1, 8, 0.1, 1, None, None) == im.IM_EINVAL
    assert L.im_estimate_spread(None, None, 0, 8, 0.1, 1, None) == im.IM_EINVAL
    assert L.im_graph_destroy(None) == im.IM_EINVAL
    assert L.im_workspace_destroy(None) == im.IM_EINVAL
    assert L.im_set_stream(None) == im.IM_OK
    assert L.im_debug_edge_hash(None, None, 0, None) == im.IM_OK
    assert L.im_debug_edge_hash(None, None, -1, None) == im.IM_EINVAL
    assert L.im_debug_lane_randoms(0, 1, None) == im.IM_EINVAL


def test_override_arguments_are_checked(L):
    for key, val in ((99, 1), (-1, 0), (im.IM_OVR_CELF_CLUSTER, 3), (im.IM_OVR_CELF_CLUSTER, 16),
                     (im.IM_OVR_UF_CAP, -2), (im.IM_OVR_FAIL_ALLOC, -1)):
        with pytest.raises(im.IMError) as e:
            im.im_debug_override(key, val)
        assert e.value.code == im.IM_EINVAL
    for key in range(im.IM_NUM_OVERRIDES):
        im.im_debug_override(key, 0)
