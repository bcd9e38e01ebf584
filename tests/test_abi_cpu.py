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


def _header_enum(prefix):
    """{NAME: value} of the `prefix*` enum constants in include/im.h."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "include", "im.h")
    with open(path) as f:
        text = f.read()
    return {m.group(1): int(m.group(2))
            for m in re.finditer(r"\b(%s[A-Z0-9_]+)\s*=\s*(-?\d+)" % prefix, text)}


def test_binding_name_tables_follow_the_header_enums():
    """The binding's per-phase and per-counter name tables line up with the
    header's indices, so profiles and work counters are read under the right
    names."""
    phases = _header_enum("IM_PHASE_")
    counts = _header_enum("IM_NUM_")
    assert len(im.PHASES) == counts["IM_NUM_PHASES"]
    for name, idx in phases.items():
        assert im.PHASES[idx] == name[len("IM_PHASE_"):].lower(), name
    stats = _header_enum("IM_STAT_")
    assert len(im.STATS) == counts["IM_NUM_STATS"]
    assert sorted(stats.values()) == list(range(len(im.STATS)))
    for name in ("IM_STAT_CHECK_CODE", "IM_STAT_SPREAD_COMPONENTS", "IM_STAT_MEMO_LIVE",
                 "IM_STAT_CELF_ROUNDS", "IM_STAT_CELF_REFRESHED"):
        assert im.STATS[stats[name]] == name[len("IM_STAT_"):].lower(), name
    server = _header_enum("IM_SERVER_STAT_")
    assert len(im.SERVER_STATS) == server.pop("IM_SERVER_STAT_COUNT")
    for name, idx in server.items():
        assert im.SERVER_STATS[idx] == name[len("IM_SERVER_STAT_"):].lower(), name
