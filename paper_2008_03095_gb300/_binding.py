"""ctypes binding of the C ABI in include/im.h (argument marshalling only).

Every function here keeps the C name and forwards to the sm_103a library
paper_2008_03095_gb300/_build/libim_gb300.so; there is no CPU fallback. If
the library has not been built, the first call raises RuntimeError.
Host arrays are numpy arrays; device arrays are torch CUDA tensors (or raw
integer device addresses).
"""
import ctypes
import os
import re

import numpy as np

from . import build as _build

IM_OK = 0
IM_EINVAL = -1
IM_ENOMEM = -2
IM_ECUDA = -3
IM_ETIMEOUT = -4
IM_EBUSY = -5
IM_EINTERNAL = -6

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "im.h")


class IMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("im error %d: %s" % (code, msg))
        self.code = code


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: build it with "
                           "paper_2008_03095_gb300.build.build(); there is no CPU fallback" % path)
    L = ctypes.CDLL(path)
    i32, i64, u32, u64, f64, P = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p)
    sig = {
        "im_graph_create": [i32, i64, P, P, P],
        "im_graph_destroy": [P],
        "im_graph_info": [P, P, P],
        "im_select_seeds": [P, i32, i32, f64, u32, P, P],
        "im_estimate_spread": [P, P, i32, i32, f64, u32, P],
        "im_estimate_spread_noalloc": [P, P, i32, i32, f64, u32, P],
        "im_workspace_create": [P, i32, P],
        "im_workspace_destroy": [P],
        "im_select_seeds_async": [P, P, i32, i32, f64, u32, P, P],
        "im_estimate_spread_async": [P, P, P, i32, i32, f64, u32, P],
        "im_workspace_status": [P],
        "im_workspace_stats": [P, P],
        "im_set_stream": [P],
        "im_sampling_threshold": [f64, P],
        "im_debug_labels": [P, i32, f64, u32, P],
        "im_debug_sizes": [P, i32, f64, u32, P],
        "im_debug_tables_lanes": [P, i32, f64, u32, P, i32, P, P],
        "im_debug_lane_randoms": [i32, u32, P],
        "im_debug_edge_hash": [P, P, i64, P],
        "im_debug_select_seeds_masked": [P, i32, i32, P, P, P, P, P],
        "im_debug_estimate_spread_masked": [P, P, i32, i32, P, P],
        "im_debug_override": [i32, i64],
        "im_graph_create_weighted": [i32, i64, P, P, P, P],
        "im_batch_create": [P, i32, P, i32, P],
        "im_batch_destroy": [P],
        "im_batch_run_async": [P],
        "im_batch_results": [P, P, P, P],
        "im_batch_query_stats": [P, i32, P],
        "im_batch_info": [P, P],
        "im_batch_phase_cycles": [P, P],
        "im_batch_autotune": [P, i32],
        "im_autotune_cache_save": [ctypes.c_char_p],
        "im_autotune_cache_load": [ctypes.c_char_p],
        "im_autotune_cache_clear": [],
        "im_server_create": [P, i32, i32, i64, P],
        "im_server_submit": [P, P, P],
        "im_server_wait": [P, u64, i64, P, P, P],
        "im_server_stats": [P, P],
        "im_server_destroy": [P],
        "im_debug_tables_ex": [P, i32, f64, u32, u32, P, P],
        "im_select_seeds_ex": [P, i32, i32, f64, u32, u32, P, P],
        "im_estimate_spread_ex": [P, P, i32, i32, f64, u32, u32, P],
        "im_select_seeds_ex_async": [P, P, i32, i32, f64, u32, u32, P, P],
        "im_estimate_spread_ex_async": [P, P, P, i32, i32, f64, u32, u32, P],
        "im_debug_first_gains": [P, i32, f64, u32, P],
        "im_profile_enable": [ctypes.c_int],
        "im_profile_read": [P, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.im_last_error.argtypes = []
    L.im_last_error.restype = ctypes.c_char_p
    L.im_kernel_launches.argtypes = []
    L.im_kernel_launches.restype = ctypes.c_uint64
    _lib = L
    return L


def header_functions():
    """Names of every function declared in include/im.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(im_\w+)\s*\(", text, re.M)))


def im_last_error():
    return lib().im_last_error().decode()


def _check(rc):
    if rc != IM_OK:
        raise IMError(rc, im_last_error())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("unsupported array type %r" % type(a))


class Graph:
    """Owning wrapper of an im_graph handle."""

    def __init__(self, handle, n, m):
        self.handle = handle
        self.n = n
        self.m = m

    def close(self):
        if self.handle:
            _check(lib().im_graph_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Workspace:
    """Owning wrapper of an im_workspace handle."""

    def __init__(self, handle, graph, R_max):
        self.handle = handle
        self.graph = graph
        self.R_max = R_max

    def close(self):
        if self.handle:
            _check(lib().im_workspace_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _gh(g):
    return g.handle if isinstance(g, Graph) else g


def im_graph_create(xadj, adj):
    xadj = np.ascontiguousarray(xadj, dtype=np.int32)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    n = xadj.shape[0] - 1
    m = adj.shape[0] // 2
    out = ctypes.c_void_p()
    _check(lib().im_graph_create(n, m, _ptr(xadj), _ptr(adj) if adj.size else None,
                                 ctypes.byref(out)))
    return Graph(out, n, m)


IM_SAMPLE_EDGE_WEIGHTS = 1
IM_SAMPLE_MIXED_HASH = 2
IM_ALGO_FUSED_SAMPLING = 4


def im_graph_create_weighted(xadj, adj, w):
    """Graph with one probability per CSR arc (float64[2m])."""
    xadj = np.ascontiguousarray(xadj, dtype=np.int32)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n = xadj.shape[0] - 1
    m = adj.shape[0] // 2
    if w.shape[0] != adj.shape[0]:
        raise ValueError("one weight per CSR arc is required")
    out = ctypes.c_void_p()
    _check(lib().im_graph_create_weighted(n, m, _ptr(xadj), _ptr(adj) if adj.size else None,
                                          _ptr(w) if w.size else None, ctypes.byref(out)))
    return Graph(out, n, m)


def im_select_seeds_ex(g, K, R, p, rng_seed, flags, out_seeds=None, out_sigma=None):
    seeds = np.empty(max(K, 0), dtype=np.int32) if out_seeds is None else out_seeds
    sigma = np.empty(max(K, 0), dtype=np.uint64) if out_sigma is None else out_sigma
    _check(lib().im_select_seeds_ex(_gh(g), K, R, p, rng_seed & 0xFFFFFFFF, flags, _ptr(seeds),
                                    _ptr(sigma)))
    return seeds, sigma


def im_estimate_spread_ex(g, seeds, R, p, rng_seed, flags):
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    out = ctypes.c_uint64()
    _check(lib().im_estimate_spread_ex(_gh(g), _ptr(seeds), seeds.shape[0], R, p,
                                       rng_seed & 0xFFFFFFFF, flags, ctypes.byref(out)))
    return int(out.value)


def im_select_seeds_ex_async(g, ws, K, R, p, rng_seed, flags, d_seeds, d_sigma):
    _check(lib().im_select_seeds_ex_async(_gh(g), ws.handle, K, R, p, rng_seed & 0xFFFFFFFF,
                                          flags, _ptr(d_seeds), _ptr(d_sigma)))


def im_estimate_spread_ex_async(g, ws, d_seeds, num_seeds, R, p, rng_seed, flags, d_sigma):
    _check(lib().im_estimate_spread_ex_async(_gh(g), ws.handle, _ptr(d_seeds), num_seeds, R, p,
                                             rng_seed & 0xFFFFFFFF, flags, _ptr(d_sigma)))


def im_graph_create_raw(n, m, xadj_ptr, adj_ptr):
    """Create from raw host addresses (e.g. pinned torch tensors)."""
    out = ctypes.c_void_p()
    _check(lib().im_graph_create(n, m, _ptr(xadj_ptr), _ptr(adj_ptr), ctypes.byref(out)))
    return Graph(out, n, m)


def im_graph_destroy(g):
    g.close()


def im_graph_info(g):
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    _check(lib().im_graph_info(_gh(g), ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def im_select_seeds(g, K, R, p, rng_seed, out_seeds=None, out_sigma=None):
    seeds = np.empty(max(K, 0), dtype=np.int32) if out_seeds is None else out_seeds
    sigma = np.empty(max(K, 0), dtype=np.uint64) if out_sigma is None else out_sigma
    _check(lib().im_select_seeds(_gh(g), K, R, p, rng_seed & 0xFFFFFFFF, _ptr(seeds), _ptr(sigma)))
    return seeds, sigma


def im_estimate_spread(g, seeds, R, p, rng_seed):
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    out = ctypes.c_uint64()
    _check(lib().im_estimate_spread(_gh(g), _ptr(seeds), seeds.shape[0], R, p,
                                    rng_seed & 0xFFFFFFFF, ctypes.byref(out)))
    return int(out.value)


def im_estimate_spread_noalloc(g, seeds, R, p, rng_seed):
    """im_estimate_spread without device allocation (static scratch; see
    NOALLOC_LIMITS for the largest n, m, R and seed count it accepts)."""
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    out = ctypes.c_uint64()
    _check(lib().im_estimate_spread_noalloc(_gh(g), _ptr(seeds), seeds.shape[0], R, p,
                                            rng_seed & 0xFFFFFFFF, ctypes.byref(out)))
    return int(out.value)


def _header_defines(prefix):
    with open(HEADER) as f:
        text = f.read()
    return {k: int(v) for k, v in re.findall(r"^#define\s+(%s\w+)\s+(\d+)" % prefix, text, re.M)}


# Limits of im_estimate_spread_noalloc, read from include/im.h.
NOALLOC_LIMITS = _header_defines("IM_NOALLOC_")


def im_workspace_create(g, R_max):
    out = ctypes.c_void_p()
    _check(lib().im_workspace_create(_gh(g), R_max, ctypes.byref(out)))
    return Workspace(out, g, R_max)


def im_workspace_destroy(ws):
    ws.close()


def im_select_seeds_async(g, ws, K, R, p, rng_seed, d_seeds, d_sigma):
    _check(lib().im_select_seeds_async(_gh(g), ws.handle, K, R, p, rng_seed & 0xFFFFFFFF,
                                       _ptr(d_seeds), _ptr(d_sigma)))


def im_estimate_spread_async(g, ws, d_seeds, num_seeds, R, p, rng_seed, d_sigma):
    _check(lib().im_estimate_spread_async(_gh(g), ws.handle, _ptr(d_seeds), num_seeds, R, p,
                                          rng_seed & 0xFFFFFFFF, _ptr(d_sigma)))


def im_workspace_status(ws):
    _check(lib().im_workspace_status(ws.handle))


STATS = ("celf_rounds", "celf_evaluations", "celf_extractions", "spread_levels",
         "celf_cycles_extract", "celf_cycles_eval", "celf_cycles_commit", "celf_cycles_merge",
         "celf_refreshes", "celf_cycles_commits", "celf_cycles_cover", "celf_refreshed",
         "celf_cycles_refresh", "check_code", "check_v0", "check_v1", "spread_components",
         "memo_accumulators", "memo_live")


def im_workspace_stats(ws):
    """{counter: value} accumulated on the device since the last call."""
    out = np.zeros(len(STATS), dtype=np.int64)
    _check(lib().im_workspace_stats(ws.handle, _ptr(out)))
    return {name: int(out[i]) for i, name in enumerate(STATS)}


def im_set_stream(stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(lib().im_set_stream(ctypes.c_void_p(stream) if stream else None))


def im_sampling_threshold(p):
    out = ctypes.c_uint64()
    _check(lib().im_sampling_threshold(p, ctypes.byref(out)))
    return int(out.value)


PHASES = ("prep", "union", "compress", "gains", "celf", "spread_prep", "spread", "spread_cc",
          "spread_union", "spread_mark")


def im_profile_enable(on=True):
    _check(lib().im_profile_enable(1 if on else 0))


def im_profile_read():
    """{phase: (total_ms, launches)} since the last enable/read."""
    ms = np.zeros(len(PHASES), dtype=np.float64)
    cnt = np.zeros(len(PHASES), dtype=np.int64)
    _check(lib().im_profile_read(_ptr(ms), _ptr(cnt)))
    return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(PHASES)}


def im_kernel_launches():
    return int(lib().im_kernel_launches())


# ------------------------------------------------------------------ test hooks


def im_debug_labels(g, R, p, rng_seed):
    out = np.empty((g.n, R), dtype=np.int32)
    _check(lib().im_debug_labels(_gh(g), R, p, rng_seed & 0xFFFFFFFF, _ptr(out)))
    return out


def im_debug_tables_lanes(g, R, p, rng_seed, lanes):
    """(labels int32[n, L], sizes uint32[n, L]) for the simulations in `lanes`."""
    lanes = np.ascontiguousarray(lanes, dtype=np.int32)
    n = g.n
    lab = np.empty((n, lanes.shape[0]), dtype=np.int32)
    siz = np.empty((n, lanes.shape[0]), dtype=np.uint32)
    _check(lib().im_debug_tables_lanes(_gh(g), R, p, rng_seed & 0xFFFFFFFF, _ptr(lanes),
                                       lanes.shape[0], _ptr(lab), _ptr(siz)))
    return lab, siz


def im_debug_first_gains(g, R, p, rng_seed):
    """uint64[n]: mg_v = sum_r |C_r(v)| as computed on the device."""
    out = np.empty(g.n, dtype=np.uint64)
    _check(lib().im_debug_first_gains(_gh(g), R, p, rng_seed & 0xFFFFFFFF, _ptr(out)))
    return out


def im_debug_tables_ex(g, R, p, rng_seed, flags):
    """(labels int32[n, R], sizes uint32[n, R]) under the IM_SAMPLE_* options."""
    lab = np.empty((g.n, R), dtype=np.int32)
    siz = np.empty((g.n, R), dtype=np.uint32)
    _check(lib().im_debug_tables_ex(_gh(g), R, p, rng_seed & 0xFFFFFFFF, flags, _ptr(lab),
                                    _ptr(siz)))
    return lab, siz


def im_debug_sizes(g, R, p, rng_seed):
    out = np.empty((g.n, R), dtype=np.uint32)
    _check(lib().im_debug_sizes(_gh(g), R, p, rng_seed & 0xFFFFFFFF, _ptr(out)))
    return out


def im_debug_lane_randoms(R, rng_seed):
    out = np.empty(R, dtype=np.uint32)
    _check(lib().im_debug_lane_randoms(R, rng_seed & 0xFFFFFFFF, _ptr(out)))
    return out


def im_debug_edge_hash(u, v):
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    out = np.empty(u.shape[0], dtype=np.uint32)
    _check(lib().im_debug_edge_hash(_ptr(u), _ptr(v), u.shape[0], _ptr(out)))
    return out


def im_debug_select_seeds_masked(g, K, mask, tables=False):
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    R = mask.shape[1]
    seeds = np.empty(max(K, 0), dtype=np.int32)
    sigma = np.empty(max(K, 0), dtype=np.uint64)
    lab = np.empty((g.n, R), dtype=np.int32) if tables else None
    siz = np.empty((g.n, R), dtype=np.uint32) if tables else None
    _check(lib().im_debug_select_seeds_masked(_gh(g), K, R, _ptr(mask), _ptr(seeds), _ptr(sigma),
                                              _ptr(lab), _ptr(siz)))
    return (seeds, sigma, lab, siz) if tables else (seeds, sigma)


IM_OVR_CELF_CLUSTER = 0
IM_OVR_CELF_ROUND_CAP = 1
IM_OVR_UF_CAP = 2
IM_OVR_SPREAD_LEVEL_CAP = 3
IM_OVR_FAIL_ALLOC = 4
IM_OVR_CELF_REFRESH_AFTER = 5
IM_OVR_BATCH_GROUP = 6
IM_OVR_CELF_EXT_REFRESH = 7
IM_NUM_OVERRIDES = 8


def im_debug_override(key, value):
    """Test-only process-wide override (IM_OVR_* key; value 0 restores the default)."""
    _check(lib().im_debug_override(key, value))


def im_debug_clear_overrides():
    for k in range(IM_NUM_OVERRIDES):
        lib().im_debug_override(k, 0)


def im_debug_estimate_spread_masked(g, seeds, mask):
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    out = ctypes.c_uint64()
    _check(lib().im_debug_estimate_spread_masked(_gh(g), _ptr(seeds), seeds.shape[0],
                                                 mask.shape[1], _ptr(mask), ctypes.byref(out)))
    return int(out.value)


# ------------------------------------------------------------------ batches


class BatchQuery(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int32), ("K", ctypes.c_int32), ("R", ctypes.c_int32),
                ("p", ctypes.c_double), ("rng_seed", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class Batch:
    """Owning wrapper of an im_batch handle; keeps its graphs alive."""

    def __init__(self, handle, graphs, Ks):
        self.handle = handle
        self.graphs = graphs
        self.Ks = list(Ks)

    def close(self):
        if self.handle:
            _check(lib().im_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def im_batch_create(graphs, queries):
    """graphs: list of Graph; queries: list of dicts with keys graph, K, R, p,
    rng_seed and optional flags."""
    n = len(queries)
    arr = (BatchQuery * n)()
    for i, q in enumerate(queries):
        arr[i] = BatchQuery(int(q["graph"]), int(q["K"]), int(q["R"]), float(q["p"]),
                            int(q["rng_seed"]) & 0xFFFFFFFF, int(q.get("flags", 0)))
    handles = (ctypes.c_void_p * len(graphs))(*[_gh(g).value if hasattr(_gh(g), "value")
                                                else _gh(g) for g in graphs])
    out = ctypes.c_void_p()
    _check(lib().im_batch_create(handles, len(graphs), arr, n, ctypes.byref(out)))
    return Batch(out, list(graphs), [int(q["K"]) for q in queries])


def im_batch_run_async(b):
    _check(lib().im_batch_run_async(b.handle))


def im_batch_results(b, check=True):
    """(list of seeds int32[K_i], list of sigmaR uint64[K_i], statuses int32[count])."""
    total = sum(b.Ks)
    seeds = np.empty(max(total, 1), dtype=np.int32)
    sigma = np.empty(max(total, 1), dtype=np.uint64)
    status = np.empty(len(b.Ks), dtype=np.int32)
    rc = lib().im_batch_results(b.handle, _ptr(seeds), _ptr(sigma), _ptr(status))
    if check:
        _check(rc)
    off = np.concatenate([[0], np.cumsum(b.Ks)])
    return ([seeds[off[i]:off[i + 1]] for i in range(len(b.Ks))],
            [sigma[off[i]:off[i + 1]] for i in range(len(b.Ks))], status)


def im_batch_query_stats(b, query):
    out = np.zeros(len(STATS), dtype=np.int64)
    _check(lib().im_batch_query_stats(b.handle, query, _ptr(out)))
    return {name: int(out[i]) for i, name in enumerate(STATS)}


BATCH_INFO = ("queries", "items", "device_bytes", "total_K", "levels", "schedule")


def im_batch_info(b):
    out = np.zeros(len(BATCH_INFO), dtype=np.int64)
    _check(lib().im_batch_info(b.handle, _ptr(out)))
    return {name: int(out[i]) for i, name in enumerate(BATCH_INFO)}


BATCH_PHASES = ("lanes", "init", "union", "compress", "gains", "celf")


def im_batch_phase_cycles(b):
    """{"wait": {phase: cycles}, "work": {phase: cycles}, "help": cycles} of the last run."""
    out = np.zeros(2 * len(BATCH_PHASES) + 1, dtype=np.int64)
    _check(lib().im_batch_phase_cycles(b.handle, _ptr(out)))
    k = len(BATCH_PHASES)
    return {"wait": dict(zip(BATCH_PHASES, out[:k].tolist())),
            "work": dict(zip(BATCH_PHASES, out[k:2 * k].tolist())), "help": int(out[2 * k])}


def im_batch_autotune(b, trials=3):
    _check(lib().im_batch_autotune(b.handle, trials))


def im_batch_destroy(b):
    b.close()


def im_autotune_cache_save(path):
    _check(lib().im_autotune_cache_save(path.encode()))


def im_autotune_cache_load(path):
    _check(lib().im_autotune_cache_load(path.encode()))


def im_autotune_cache_clear():
    _check(lib().im_autotune_cache_clear())


# ------------------------------------------------------------------ serving

IM_REQUEST_SELECT = 0
IM_REQUEST_SPREAD = 1


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("graph", ctypes.c_int32), ("K", ctypes.c_int32),
                ("R", ctypes.c_int32), ("p", ctypes.c_double), ("rng_seed", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("seeds", ctypes.c_void_p)]


class Server:
    """Owning wrapper of an im_server handle; keeps its graphs alive."""

    def __init__(self, handle, graphs):
        self.handle = handle
        self.graphs = graphs
        self.kinds = {}

    def close(self):
        if self.handle:
            _check(lib().im_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def im_server_create(graphs, slots=8, memory_budget=64 << 30):
    handles = (ctypes.c_void_p * len(graphs))(*[_gh(g).value if hasattr(_gh(g), "value")
                                                else _gh(g) for g in graphs])
    out = ctypes.c_void_p()
    _check(lib().im_server_create(handles, len(graphs), slots, int(memory_budget),
                                  ctypes.byref(out)))
    return Server(out, list(graphs))


def im_server_submit(sv, kind, graph, K, R, p, rng_seed, flags=0, seeds=None):
    """Queue a query; returns its ticket. spread: seeds is the seed set (K = len)."""
    arr = None
    if kind == IM_REQUEST_SPREAD:
        arr = np.ascontiguousarray(seeds if seeds is not None else [], dtype=np.int32)
        K = arr.shape[0]
    req = Request(kind, graph, K, R, float(p), rng_seed & 0xFFFFFFFF, flags,
                  arr.ctypes.data if arr is not None and arr.size else None)
    t = ctypes.c_uint64()
    _check(lib().im_server_submit(sv.handle, ctypes.byref(req), ctypes.byref(t)))
    sv.kinds[t.value] = (kind, K)
    return t.value


def im_server_wait(sv, ticket, timeout_us=-1):
    """select: (seeds, sigma, times); spread: (None, sigmaR, times). times =
    (submitted, admitted, done) in seconds since the server started. Raises
    IMError(IM_EBUSY) if not done within timeout_us (0 = poll)."""
    kind, K = sv.kinds[ticket]
    seeds = np.empty(max(K, 1), dtype=np.int32)
    sigma = np.empty(max(K, 1), dtype=np.uint64)
    times = np.zeros(3, dtype=np.float64)
    rc = lib().im_server_wait(sv.handle, ticket, int(timeout_us), _ptr(seeds), _ptr(sigma),
                              _ptr(times))
    if rc != IM_EBUSY:
        sv.kinds.pop(ticket, None)
    _check(rc)
    if kind == IM_REQUEST_SELECT:
        return seeds[:K], sigma[:K], tuple(times)
    return None, int(sigma[0]), tuple(times)


SERVER_STATS = ("submitted", "admitted", "completed", "in_flight", "in_flight_peak", "queued",
                "queue_peak", "ws_created", "ws_evicted", "pool_bytes", "pool_bytes_peak",
                "budget")


def im_server_stats(sv):
    out = np.zeros(len(SERVER_STATS), dtype=np.int64)
    _check(lib().im_server_stats(sv.handle, _ptr(out)))
    return {name: int(out[i]) for i, name in enumerate(SERVER_STATS)}


def im_server_destroy(sv):
    sv.close()
