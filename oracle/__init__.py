"""CPU oracle for fused-sampling influence maximization (arXiv 2008.03095).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only users. The product path never
imports this module. The oracle is a slow, literal C++ restatement of the
method (Section 3.1 Eq. 1-2, Algorithms 1, 4, 5 and 7 on fixed samples); see
im_oracle.cpp for the definition of every quantity.

Every function takes and returns numpy arrays (host memory) and raises
ValueError when the oracle rejects its input.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_libs = {}
_variant = "single"


def use_all_cores(on: bool = True):
    """Switch every following call to the OpenMP build (all host cores, or
    OMP_NUM_THREADS) or back to the single-threaded default. Both builds give
    identical results."""
    global _variant
    _variant = "omp" if on else "single"


def threads():
    """Threads the current build uses (1 for the single-threaded build)."""
    if _variant != "omp":
        return 1
    return int(lib().orc_max_threads())


def lib():
    L = _libs.get(_variant)
    if L is None:
        path = _build.build_omp() if _variant == "omp" else _build.build()
        L = ctypes.CDLL(path)
        i32, i64, u32, u64, f64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
        P = ctypes.c_void_p
        L.orc_murmur3_x86_32.argtypes = [P, i32, u32]
        L.orc_murmur3_x86_32.restype = u32
        L.orc_edge_hash.argtypes = [i32, i32]
        L.orc_edge_hash.restype = u32
        L.orc_mt19937.argtypes = [u32, i64, P]
        L.orc_mt19937.restype = None
        L.orc_threshold.argtypes = [f64]
        L.orc_threshold.restype = u64
        L.orc_live.argtypes = [i32, i32, u32, f64]
        L.orc_live.restype = i32
        L.orc_validate_csr.argtypes = [i32, i64, P, P]
        L.orc_validate_csr.restype = i32
        L.orc_labels.argtypes = [i32, i64, P, P, i32, f64, u32, P, P]
        L.orc_labels.restype = i32
        L.orc_labels_lanes.argtypes = [i32, i64, P, P, i32, f64, u32, i32, P, P, P]
        L.orc_labels_lanes.restype = i32
        L.orc_select_seeds.argtypes = [i32, i64, P, P, i32, i32, f64, u32, P, P]
        L.orc_select_seeds.restype = i32
        L.orc_estimate_spread.argtypes = [i32, i64, P, P, P, i32, i32, f64, u32, P]
        L.orc_estimate_spread.restype = i32
        L.orc_greedy_from_tables.argtypes = [i32, i32, P, P, i32, P, P]
        L.orc_greedy_from_tables.restype = i32
        L.orc_marginal_gains.argtypes = [i32, i32, P, P, P, i32, P]
        L.orc_marginal_gains.restype = i32
        L.orc_labels_masked.argtypes = [i32, i64, P, P, i32, P, P, P]
        L.orc_labels_masked.restype = i32
        L.orc_select_seeds_masked.argtypes = [i32, i64, P, P, i32, i32, P, P, P]
        L.orc_select_seeds_masked.restype = i32
        L.orc_estimate_spread_masked.argtypes = [i32, i64, P, P, P, i32, i32, P, P]
        L.orc_estimate_spread_masked.restype = i32
        L.orc_labels_ex.argtypes = [i32, i64, P, P, i32, f64, u32, P, i32, P, P]
        L.orc_labels_ex.restype = i32
        L.orc_select_seeds_ex.argtypes = [i32, i64, P, P, i32, i32, f64, u32, P, i32, P, P]
        L.orc_select_seeds_ex.restype = i32
        L.orc_estimate_spread_ex.argtypes = [i32, i64, P, P, P, i32, i32, f64, u32, P, i32, P]
        L.orc_estimate_spread_ex.restype = i32
        L.orc_live_ex.argtypes = [i32, i32, u32, f64, f64, i32, i32]
        L.orc_live_ex.restype = i32
        L.orc_fmix32.argtypes = [u32]
        L.orc_fmix32.restype = u32
        L.orc_edge_code.argtypes = [f64]
        L.orc_edge_code.restype = u32
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = i32
        _libs[_variant] = L
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(xadj, adj):
    xadj = np.ascontiguousarray(xadj, dtype=np.int32)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    n = xadj.shape[0] - 1
    m = adj.shape[0] // 2
    return n, m, xadj, adj


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle rejected input to " + what)


def murmur3_x86_32(data: bytes, seed: int = 0) -> int:
    buf = np.frombuffer(bytes(data) + b"\0", dtype=np.uint8)
    return int(lib().orc_murmur3_x86_32(_p(buf), len(data), seed & 0xFFFFFFFF))


def edge_hash(u: int, v: int) -> int:
    return int(lib().orc_edge_hash(u, v))


def mt19937(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint32)
    lib().orc_mt19937(seed & 0xFFFFFFFF, count, _p(out))
    return out


def threshold(p: float) -> int:
    return int(lib().orc_threshold(p))


def live(u: int, v: int, x: int, p: float) -> bool:
    return bool(lib().orc_live(u, v, x & 0xFFFFFFFF, p))


def validate_csr(xadj, adj) -> bool:
    n, m, xadj, adj = _csr(xadj, adj)
    if n < 1 or adj.shape[0] % 2:
        return False
    return lib().orc_validate_csr(n, m, _p(xadj), _p(adj)) == 0


def labels(xadj, adj, R, p, seed):
    """(labels, sizes), each n x R (vertex-major), hash sampler."""
    n, m, xadj, adj = _csr(xadj, adj)
    lab = np.empty((n, R), dtype=np.int32)
    siz = np.empty((n, R), dtype=np.uint32)
    _check(lib().orc_labels(n, m, _p(xadj), _p(adj), R, p, seed, _p(lab), _p(siz)), "labels")
    return lab, siz


def labels_lanes(xadj, adj, R, p, seed, lanes):
    """(labels, sizes) for the simulations listed in `lanes`: n x len(lanes)."""
    n, m, xadj, adj = _csr(xadj, adj)
    lanes = np.ascontiguousarray(lanes, dtype=np.int32)
    nl = lanes.shape[0]
    lab = np.empty((n, nl), dtype=np.int32)
    siz = np.empty((n, nl), dtype=np.uint32)
    _check(lib().orc_labels_lanes(n, m, _p(xadj), _p(adj), R, p, seed, nl, _p(lanes), _p(lab),
                                  _p(siz)), "labels_lanes")
    return lab, siz


def select_seeds(xadj, adj, K, R, p, seed):
    """(seeds int32[K], sigmaR uint64[K]) by greedy over the R fixed samples."""
    n, m, xadj, adj = _csr(xadj, adj)
    seeds = np.empty(K, dtype=np.int32)
    sigma = np.empty(K, dtype=np.uint64)
    _check(lib().orc_select_seeds(n, m, _p(xadj), _p(adj), K, R, p, seed, _p(seeds), _p(sigma)),
           "select_seeds")
    return seeds, sigma


def estimate_spread(xadj, adj, seeds, R, p, seed) -> int:
    n, m, xadj, adj = _csr(xadj, adj)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    out = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_estimate_spread(n, m, _p(xadj), _p(adj), _p(seeds), seeds.shape[0], R, p,
                                     seed, _p(out)), "estimate_spread")
    return int(out[0])


def greedy_from_tables(lab, siz, K):
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    siz = np.ascontiguousarray(siz, dtype=np.uint32)
    n, R = lab.shape
    seeds = np.empty(K, dtype=np.int32)
    sigma = np.empty(K, dtype=np.uint64)
    _check(lib().orc_greedy_from_tables(n, R, _p(lab), _p(siz), K, _p(seeds), _p(sigma)),
           "greedy_from_tables")
    return seeds, sigma


def marginal_gains(lab, siz, S):
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    siz = np.ascontiguousarray(siz, dtype=np.uint32)
    S = np.ascontiguousarray(S, dtype=np.int32)
    n, R = lab.shape
    g = np.empty(n, dtype=np.uint64)
    _check(lib().orc_marginal_gains(n, R, _p(lab), _p(siz), _p(S), S.shape[0], _p(g)),
           "marginal_gains")
    return g


def labels_masked(xadj, adj, mask):
    """mask: uint8 [2m, R], mask[a, r] = arc a live in sample r (symmetric)."""
    n, m, xadj, adj = _csr(xadj, adj)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    R = mask.shape[1]
    lab = np.empty((n, R), dtype=np.int32)
    siz = np.empty((n, R), dtype=np.uint32)
    _check(lib().orc_labels_masked(n, m, _p(xadj), _p(adj), R, _p(mask), _p(lab), _p(siz)),
           "labels_masked")
    return lab, siz


def select_seeds_masked(xadj, adj, K, mask):
    n, m, xadj, adj = _csr(xadj, adj)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    R = mask.shape[1]
    seeds = np.empty(K, dtype=np.int32)
    sigma = np.empty(K, dtype=np.uint64)
    _check(lib().orc_select_seeds_masked(n, m, _p(xadj), _p(adj), K, R, _p(mask), _p(seeds),
                                         _p(sigma)), "select_seeds_masked")
    return seeds, sigma


def estimate_spread_masked(xadj, adj, seeds, mask) -> int:
    n, m, xadj, adj = _csr(xadj, adj)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    R = mask.shape[1]
    out = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_estimate_spread_masked(n, m, _p(xadj), _p(adj), _p(seeds), seeds.shape[0],
                                            R, _p(mask), _p(out)), "estimate_spread_masked")
    return int(out[0])


# ------------------------------------------------------------------ sampling options
# weights: None for the uniform p, else float64[2m], one probability w(u,v)
# per CSR arc (equal on both arcs of an edge); mix: the mixed-hash variant.


def _w(weights):
    if weights is None:
        return None, None
    w = np.ascontiguousarray(weights, dtype=np.float64)
    return w, _p(w)


def fmix32(h: int) -> int:
    return int(lib().orc_fmix32(h & 0xFFFFFFFF))


def edge_code(w: float) -> int:
    """32-bit threshold code of an edge probability (0xFFFFFFFF = always live)."""
    return int(lib().orc_edge_code(w))


def live_ex(u, v, x, p=0.0, w=None, mix=False) -> bool:
    return bool(lib().orc_live_ex(u, v, x & 0xFFFFFFFF, p, 0.0 if w is None else w,
                                  0 if w is None else 1, 1 if mix else 0))


def labels_ex(xadj, adj, R, p, seed, weights=None, mix=False):
    n, m, xadj, adj = _csr(xadj, adj)
    w, wp = _w(weights)
    lab = np.empty((n, R), dtype=np.int32)
    siz = np.empty((n, R), dtype=np.uint32)
    _check(lib().orc_labels_ex(n, m, _p(xadj), _p(adj), R, p, seed, wp, 1 if mix else 0,
                               _p(lab), _p(siz)), "labels_ex")
    return lab, siz


def select_seeds_ex(xadj, adj, K, R, p, seed, weights=None, mix=False):
    n, m, xadj, adj = _csr(xadj, adj)
    w, wp = _w(weights)
    seeds = np.empty(K, dtype=np.int32)
    sigma = np.empty(K, dtype=np.uint64)
    _check(lib().orc_select_seeds_ex(n, m, _p(xadj), _p(adj), K, R, p, seed, wp,
                                     1 if mix else 0, _p(seeds), _p(sigma)), "select_seeds_ex")
    return seeds, sigma


def estimate_spread_ex(xadj, adj, seeds, R, p, seed, weights=None, mix=False) -> int:
    n, m, xadj, adj = _csr(xadj, adj)
    w, wp = _w(weights)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    out = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_estimate_spread_ex(n, m, _p(xadj), _p(adj), _p(seeds), seeds.shape[0], R,
                                        p, seed, wp, 1 if mix else 0, _p(out)),
           "estimate_spread_ex")
    return int(out[0])
