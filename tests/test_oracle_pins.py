"""Pins of the CPU oracle against facts that do not come from the oracle itself:
published hash/generator reference values, the paper's worked example,
closed forms, library routines (scipy), brute force and exact invariants."""
import itertools
import math
import struct
from fractions import Fraction

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from paper_2008_03095_gb300 import synth
from tests import _util

# ------------------------------------------------------------------ hash, Eq. 1


def test_murmur3_published_vectors():
    n = 0
    for key_hex, seed_hex, exp_hex in _util.golden_lines("murmur3_x86_32_vectors.txt"):
        key = b"" if key_hex == "-" else bytes.fromhex(key_hex)
        assert oracle.murmur3_x86_32(key, int(seed_hex, 16)) == int(exp_hex, 16), key_hex
        n += 1
    assert n >= 20


def test_murmur3_smhasher_verification_value():
    key = bytes(range(256))
    hashes = b"".join(struct.pack("<I", oracle.murmur3_x86_32(key[:i], 256 - i))
                      for i in range(256))
    assert oracle.murmur3_x86_32(hashes, 0) == 0xB0F57EE3


def test_edge_hash_direction_oblivious_and_key_layout():
    rng = np.random.default_rng(0)
    for _ in range(500):
        u, v = (int(x) for x in rng.integers(0, 2 ** 31 - 1, size=2))
        h = oracle.edge_hash(u, v)
        assert h == oracle.edge_hash(v, u)
        assert h == oracle.murmur3_x86_32(struct.pack("<II", min(u, v), max(u, v)), 0)


# ------------------------------------------------------------------ X_r generator


def test_mt19937_standard_required_value():
    (seed, idx, val), = [tuple(int(t) for t in row)
                         for row in _util.golden_lines("mt19937_standard.txt")]
    assert oracle.mt19937(seed, idx)[-1] == val


@pytest.mark.parametrize("seed", [7, 1, 5489, 2 ** 32 - 1])
def test_mt19937_matches_numpy_legacy_generator(seed):
    # numpy's legacy RandomState seeds MT19937 with the same init_genrand
    # routine; its raw 32-bit outputs are an independent implementation.
    raw = np.random.RandomState(seed)._bit_generator.random_raw(3000).astype(np.uint32)
    assert np.array_equal(oracle.mt19937(seed, 3000), raw)


# ------------------------------------------------------------------ sampling, Eq. 2


def test_threshold_closed_forms():
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(1.0) == 2 ** 32
    assert oracle.threshold(0.5) == 2 ** 31
    assert oracle.threshold(0.01) == 42949672  # floor(42949672.96)
    assert oracle.threshold(2.0 ** -32) == 1


def test_live_rate_matches_threshold():
    rng = np.random.default_rng(3)
    for p in (0.01, 0.05, 0.3):
        hits = 0
        N = 20000
        for _ in range(N):
            u, v = (int(x) for x in rng.integers(0, 10 ** 6, size=2))
            x = int(rng.integers(0, 2 ** 32))
            hits += oracle.live(u, v, x, p)
        se = math.sqrt(p * (1 - p) / N)
        assert abs(hits / N - p) < 5 * se


def test_live_extremes():
    rng = np.random.default_rng(4)
    for _ in range(200):
        u, v, x = int(rng.integers(0, 1000)), int(rng.integers(0, 1000)), int(rng.integers(0, 2 ** 32))
        assert not oracle.live(u, v, x, 0.0)
        assert oracle.live(u, v, x, 1.0)


# ------------------------------------------------------------------ worked example


def test_worked_example_figures_3_4():
    xadj, adj, mask, exp = _util.worked_example()
    lab, siz = oracle.labels_masked(xadj, adj, mask)
    assert np.array_equal(lab, exp["labels"])
    # size memo: sample 1 {A:4, B:1}, sample 2 {A:5}; zero off the roots
    want = np.zeros((5, 2), dtype=np.uint32)
    want[0, 0], want[1, 0], want[0, 1] = 4, 1, 5
    assert np.array_equal(siz, want)
    mg = [int(sum(siz[lab[v, r], r] for r in range(2))) for v in range(5)]
    assert mg == exp["mg"]
    seeds, sigma = oracle.select_seeds_masked(xadj, adj, 1, mask)
    assert int(seeds[0]) == exp["first_seed"] and int(sigma[0]) == exp["first_sigmaR"]
    assert oracle.estimate_spread_masked(xadj, adj, [exp["first_seed"]], mask) == 9


# ------------------------------------------------------------------ closed forms


def _cc_min_labels(n, edges):
    if not edges:
        return np.arange(n)
    e = np.array(edges)
    g = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    mins = np.full(comp.max() + 1, n)
    np.minimum.at(mins, comp, np.arange(n))
    return mins[comp]


def test_p0_closed_form():
    xadj, adj = synth.chung_lu(300, 900, 2.5, 11)
    R, K = 37, 12
    lab, siz = oracle.labels(xadj, adj, R, 0.0, 7)
    assert np.array_equal(lab, np.repeat(np.arange(300)[:, None], R, axis=1))
    assert np.all(siz == 1)
    seeds, sigma = oracle.select_seeds(xadj, adj, K, R, 0.0, 7)
    assert list(seeds) == list(range(K))
    assert list(sigma) == [R * (k + 1) for k in range(K)]
    assert oracle.estimate_spread(xadj, adj, [5, 9, 5], R, 0.0, 7) == 2 * R


def test_p1_closed_form():
    # a graph with several components of different sizes
    n = 120
    rng = np.random.default_rng(5)
    parts = np.split(rng.permutation(n), [50, 80, 100, 110, 115])
    edges = set()
    for part in parts:
        part = list(part)
        for i in range(1, len(part)):  # spanning path + random chords
            edges.add(tuple(sorted((part[i - 1], part[i]))))
        for _ in range(len(part)):
            a, b = rng.choice(part, 2)
            if a != b:
                edges.add(tuple(sorted((a, b))))
    edges = sorted(edges)
    xadj, adj = synth.csr_from_edges(n, [e[0] for e in edges], [e[1] for e in edges])
    R = 5
    lab, siz = oracle.labels(xadj, adj, R, 1.0, 3)
    cc = _cc_min_labels(n, edges)
    for r in range(R):
        assert np.array_equal(lab[:, r], cc)
    csize = np.bincount(cc, minlength=n)
    assert np.array_equal(siz[:, 0], csize.astype(np.uint32))
    # greedy: largest uncovered component first (its smallest id), ties by id,
    # then zero-gain vertices in id order
    K = 9
    seeds, sigma = oracle.select_seeds(xadj, adj, K, R, 1.0, 3)
    roots = sorted(set(cc.tolist()), key=lambda c: (-csize[c], c))
    want, tot, wsig = [], 0, []
    for c in roots:
        want.append(c)
        tot += R * int(csize[c])
        wsig.append(tot)
    rest = [v for v in range(n) if v not in want]
    while len(want) < K:
        want.append(rest.pop(0))
        wsig.append(tot)
    assert list(seeds) == want[:K] and list(sigma) == wsig[:K]
    assert oracle.estimate_spread(xadj, adj, want[:3], R, 1.0, 3) == wsig[2]


# ------------------------------------------------------------------ library routine


@pytest.mark.parametrize("p", [0.05, 0.2, 0.5])
def test_labels_match_scipy_and_union_find(p):
    xadj, adj = synth.chung_lu(400, 1600, 2.3, 21)
    R, seed = 24, 99
    lab, siz = oracle.labels(xadj, adj, R, p, seed)
    X = np.random.RandomState(seed)._bit_generator.random_raw(R).astype(np.uint64)
    T = math.floor(p * 2 ** 32)
    edges = _util.edge_list(xadj, adj)
    h = np.array([oracle.edge_hash(u, v) for u, v in edges], dtype=np.uint64)
    for r in range(R):
        live_edges = [e for e, hv in zip(edges, h) if (int(X[r]) ^ int(hv)) < T]
        want = _cc_min_labels(400, live_edges)
        assert np.array_equal(lab[:, r], want)
        assert np.array_equal(lab[:, r], _util.uf_min_labels(400, live_edges))
        counts = np.bincount(want, minlength=400)
        assert np.array_equal(siz[:, r], counts.astype(np.uint32))


# ------------------------------------------------------------------ invariants


def test_size_table_invariants():
    xadj, adj = synth.chung_lu(500, 2500, 2.2, 8)
    R = 40
    lab, siz = oracle.labels(xadj, adj, R, 0.1, 1)
    assert np.all(siz.sum(axis=0, dtype=np.int64) == 500)
    is_root = lab == np.arange(500)[:, None]
    assert np.all(siz[~is_root] == 0) and np.all(siz[is_root] > 0)
    # sizes indexed through labels equal component sizes
    for r in range(R):
        assert np.array_equal(siz[lab[:, r], r], np.bincount(lab[:, r], minlength=500)[lab[:, r]])


def test_bfs_spread_equals_count_of_slots_sharing_a_seed_label():
    """sigma*R (Algorithm 4's BFS over the samples) equals the number of
    (vertex, sample) slots whose component label is some seed's label: the
    identity the spread's hand-over counts on, taken here between two
    independent oracle routines (BFS and union-find labels)."""
    xadj, adj = synth.chung_lu(400, 1600, 2.2, 12)
    R, p, seed = 48, 0.12, 9
    lab, _ = oracle.labels(xadj, adj, R, p, seed)
    rng = np.random.default_rng(4)
    for k in (1, 3, 9):
        S = rng.choice(400, size=k, replace=False)
        S = np.concatenate([S, S[:1]])  # a duplicate seed changes nothing
        count = sum(int(np.isin(lab[:, r], lab[S, r]).sum()) for r in range(R))
        assert count == oracle.estimate_spread(xadj, adj, [int(x) for x in S], R, p, seed)


def test_spread_monotone_and_submodular_exactly():
    xadj, adj = synth.chung_lu(200, 700, 2.4, 31)
    R, p, seed = 64, 0.15, 5
    rng = np.random.default_rng(6)

    def sig(S):
        return oracle.estimate_spread(xadj, adj, list(S), R, p, seed)

    for _ in range(40):
        T = set(int(x) for x in rng.choice(200, size=8, replace=False))
        S = set(list(T)[:3])
        v = int(rng.choice([x for x in range(200) if x not in T]))
        dS = sig(S | {v}) - sig(S)
        dT = sig(T | {v}) - sig(T)
        assert dS >= dT >= 0
        assert sig(T) >= sig(S)


def test_greedy_steps_maximize_bfs_marginal_gain():
    # The label-table greedy must pick, at every step, the vertex that maximizes
    # sigma(S + v) computed by BFS (independent code path), lowest id on ties.
    xadj, adj = synth.chung_lu(60, 150, 2.3, 41)
    R, p, seed, K = 32, 0.2, 11, 6
    seeds, sigma = oracle.select_seeds(xadj, adj, K, R, p, seed)
    S = []
    for k in range(K):
        base = oracle.estimate_spread(xadj, adj, S, R, p, seed) if S else 0
        gains = [oracle.estimate_spread(xadj, adj, S + [v], R, p, seed) - base
                 if v not in S else -1 for v in range(60)]
        best = int(np.argmax(gains))  # argmax returns the first (lowest id)
        assert seeds[k] == best
        assert sigma[k] == base + gains[best]
        S.append(best)
    assert oracle.estimate_spread(xadj, adj, list(seeds), R, p, seed) == sigma[-1]


def test_greedy_within_one_minus_one_over_e_of_brute_force_opt():
    xadj, adj = synth.random_graph(11, 18, 77)
    R, p, seed, K = 48, 0.25, 2, 3
    seeds, sigma = oracle.select_seeds(xadj, adj, K, R, p, seed)
    opt = max(oracle.estimate_spread(xadj, adj, list(c), R, p, seed)
              for c in itertools.combinations(range(11), K))
    assert sigma[-1] <= opt
    assert sigma[-1] >= (1 - 1 / math.e) * opt


def test_marginal_gains_consistent_with_greedy():
    xadj, adj = synth.chung_lu(150, 500, 2.4, 12)
    R = 16
    lab, siz = oracle.labels(xadj, adj, R, 0.1, 4)
    seeds, sigma = oracle.greedy_from_tables(lab, siz, 5)
    for k in range(5):
        g = oracle.marginal_gains(lab, siz, seeds[:k])
        assert int(np.argmax(g)) == seeds[k]
        assert int(g[seeds[k]]) == int(sigma[k]) - (int(sigma[k - 1]) if k else 0)


# ------------------------------------------------------------------ brute force


def _small_graph():
    edges = [(0, 1), (1, 2), (2, 3), (0, 3), (1, 4), (4, 5), (5, 6), (2, 6), (6, 7), (0, 7)]
    xadj, adj = synth.csr_from_edges(8, [e[0] for e in edges], [e[1] for e in edges])
    return xadj, adj, edges


def test_spread_over_all_live_subsets_matches_enumeration():
    # Lanes = all 2^m live-edge subsets: sigmaR equals the brute-force sum of
    # reach(S) over every subgraph, i.e. 2^m times the exact IC spread at p=1/2.
    xadj, adj, edges = _small_graph()
    m = len(edges)
    R = 2 ** m
    idx = {e: i for i, e in enumerate(edges)}
    mask = _util.arc_mask(xadj, adj, lambda u, v, r: (r >> idx[tuple(sorted((u, v)))]) & 1, R)
    for S in ([0], [3, 5], [1, 6, 7]):
        total = sum(len(_util.py_reach(8, [e for i, e in enumerate(edges) if (sub >> i) & 1], S))
                    for sub in range(R))
        assert oracle.estimate_spread_masked(xadj, adj, S, mask) == total
    lab, siz = oracle.labels_masked(xadj, adj, mask)
    for sub in range(0, R, 37):
        live_edges = [e for i, e in enumerate(edges) if (sub >> i) & 1]
        assert np.array_equal(lab[:, sub], _util.uf_min_labels(8, live_edges))


def _exact_hash_expectation(edges, hashes, T, n, S):
    """E over X uniform in [0, 2^32) of |reach_X(S)| (rational) and E of its square."""
    bounds = {0, 2 ** 32}
    for h in hashes:
        for i in range(32):
            if (T >> i) & 1:
                base = ((((h ^ T) >> (i + 1)) << (i + 1)) | (h & (1 << i)))
                bounds.add(base)
                bounds.add(base + (1 << i))
    b = sorted(bounds)
    e1 = Fraction(0)
    e2 = Fraction(0)
    for lo, hi in zip(b[:-1], b[1:]):
        live_edges = [e for e, h in zip(edges, hashes) if (lo ^ h) < T]
        reach = len(_util.py_reach(n, live_edges, S))
        e1 += Fraction(hi - lo, 2 ** 32) * reach
        e2 += Fraction(hi - lo, 2 ** 32) * reach * reach
    return e1, e2


@pytest.mark.parametrize("p", [0.3, 0.6])
def test_hash_sampler_expectation_by_interval_decomposition(p):
    xadj, adj, edges = _small_graph()
    T = math.floor(p * 2 ** 32)
    hashes = [oracle.edge_hash(u, v) for u, v in edges]
    S = [0, 5]
    e1, e2 = _exact_hash_expectation(edges, hashes, T, 8, S)
    R = 20000
    est = Fraction(oracle.estimate_spread(xadj, adj, S, R, p, 13), R)
    sd = math.sqrt(float(e2 - e1 * e1))
    assert abs(float(est - e1)) <= 5 * sd / math.sqrt(R)
    # The independent-edge IC value differs (edges share X_r); it is reported,
    # not asserted.
    m = len(edges)
    ic = sum((p ** bin(sub).count("1")) * ((1 - p) ** (m - bin(sub).count("1"))) *
             len(_util.py_reach(8, [e for i, e in enumerate(edges) if (sub >> i) & 1], S))
             for sub in range(2 ** m))
    print("hash-scheme E=%.4f  independent IC=%.4f" % (float(e1), ic))


# ------------------------------------------------------------------ validation


def test_oracle_rejects_invalid_csr():
    xadj, adj = synth.chung_lu(50, 120, 2.5, 2)
    assert oracle.validate_csr(xadj, adj)
    bad = adj.copy()
    bad[3] = 50  # out of range
    assert not oracle.validate_csr(xadj, bad)
    # asymmetric: drop one reverse arc by redirecting it
    x2 = np.array([0, 1, 1, 2], dtype=np.int32)
    a2 = np.array([1, 1], dtype=np.int32)  # 0->1 and 2->1, but 1 has no arcs
    assert not oracle.validate_csr(x2, a2)
    x3 = xadj.copy()
    x3[5] = x3[6] + 1  # non-monotone
    assert not oracle.validate_csr(x3, adj)
    with pytest.raises(ValueError):
        oracle.select_seeds(xadj, adj, 51, 8, 0.1, 1)  # K > n
    with pytest.raises(ValueError):
        oracle.select_seeds(xadj, adj, 3, 8, 1.5, 1)  # p > 1


@pytest.mark.parametrize("p", [0.02, 0.2])
def test_lane_sharding_invariance_of_gains_and_greedy(p):
    # Samples are independent, so lane ranges [0, R1) and [R1, R) can be
    # processed apart: their tables equal the matching columns of the full
    # tables, marginal gains are sums over the shards, and a greedy that sums
    # the shards' gains before each deterministic commit (gain desc, id asc)
    # picks the same seeds and sigma*R as the single-range greedy.
    xadj, adj = synth.chung_lu(150, 500, 2.3, 17)
    n, R, seed, K = 150, 37, 9, 8
    full_lab, full_siz = oracle.labels(xadj, adj, R, p, seed)
    shards = [np.arange(0, 13), np.arange(13, R)]
    tabs = [oracle.labels_lanes(xadj, adj, R, p, seed, lanes) for lanes in shards]
    for lanes, (lab, siz) in zip(shards, tabs):
        assert np.array_equal(lab, full_lab[:, lanes])
        assert np.array_equal(siz, full_siz[:, lanes])
    seeds, sigma = oracle.select_seeds(xadj, adj, K, R, p, seed)
    S, total = [], 0
    for k in range(K):
        g = sum(oracle.marginal_gains(lab, siz, S).astype(np.int64) for lab, siz in tabs)
        assert np.array_equal(g, oracle.marginal_gains(full_lab, full_siz, S).astype(np.int64))
        g[S] = -1
        best = int(np.argmax(g))
        total += int(g[best])
        assert seeds[k] == best and int(sigma[k]) == total
        S.append(best)


# ------------------------------------------------------------------ OpenMP build


@pytest.mark.parametrize("mk,K,R,p", [
    (lambda: synth.chung_lu(3000, 12000, 2.2, 21), 20, 96, 0.05),
    (lambda: synth.random_graph(400, 1600, 22), 30, 33, 0.3),
    (lambda: synth.chung_lu(1500, 9000, 2.1, 23), 15, 256, 0.0),
])
def test_all_core_build_gives_identical_results(mk, K, R, p):
    """The OpenMP build (all-core CPU baseline, writer of the stored expected
    values) splits simulations and greedy candidates over threads; ties must
    still go to the lowest id, so its output equals the single-threaded one."""
    xadj, adj = mk()
    want = oracle.select_seeds(xadj, adj, K, R, p, 7)
    wlab = oracle.labels(xadj, adj, R, p, 7)
    oracle.use_all_cores(True)
    try:
        assert oracle.threads() >= 1
        got = oracle.select_seeds(xadj, adj, K, R, p, 7)
        glab = oracle.labels(xadj, adj, R, p, 7)
    finally:
        oracle.use_all_cores(False)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert np.array_equal(glab[0], wlab[0]) and np.array_equal(glab[1], wlab[1])


def test_stored_expected_values_match_the_committed_graph_digests():
    """Rows of tests/golden/oracle_expected_seeds.txt name the graph they ran
    on; the digests must be the committed ones, K and R the workload's, and
    sigma*R a non-decreasing sequence with positive first entry."""
    import sys
    sys.path.insert(0, _util.GOLDEN)
    from make_oracle_expected import read_expected

    digests = {row[0]: row[4] for row in _util.golden_lines("graph_sha256.txt")}
    exp = read_expected()
    assert {k[0] for k in exp} >= {"clustered_n334863", "powerlaw_n4m"}
    for (name, p), (sha, K, R, seed, seeds, sigma) in exp.items():
        w = synth.WORKLOADS[name]
        assert sha == digests[name]
        assert (K, R, seed) == (w["K"], w["R"], w["rng_seed"]) and p in w["ps"]
        assert len(set(seeds.tolist())) == K and len(sigma) == K
        assert sigma[0] > 0 and np.all(np.diff(sigma.astype(np.int64)) >= 0)


# ------------------------------------------------------------------ per-edge weights, mixed hash


def test_fmix32_is_murmur3_of_the_empty_key():
    """MurmurHash3 of an empty key is the finalizer applied to the seed, so the
    published empty-key vectors pin fmix32 (and fmix32 is a bijection)."""
    for key_hex, seed_hex, exp_hex in _util.golden_lines("murmur3_x86_32_vectors.txt"):
        if key_hex == "-":
            assert oracle.fmix32(int(seed_hex, 16)) == int(exp_hex, 16)
    xs = np.random.default_rng(3).integers(0, 2 ** 32, size=20000, dtype=np.uint64)
    assert len({oracle.fmix32(int(x)) for x in xs}) == len(set(xs.tolist()))


def test_edge_codes_closed_forms():
    assert oracle.edge_code(0.0) == 0
    assert oracle.edge_code(1.0) == 0xFFFFFFFF
    assert oracle.edge_code(0.5) == 2 ** 31
    assert oracle.edge_code(2.0 ** -32) == 1
    for p in (0.01, 0.05, 0.3, 0.999):
        assert oracle.edge_code(p) == oracle.threshold(p)
    u, v = 3, 9
    for x in (0, 1, 12345, 2 ** 32 - 1):
        assert not oracle.live_ex(u, v, x, w=0.0)
        assert oracle.live_ex(u, v, x, w=1.0)
        assert oracle.live_ex(u, v, x, p=0.01, w=0.01) == oracle.live(u, v, x, 0.01)
        assert not oracle.live_ex(u, v, x, p=0.0, mix=True)
        assert oracle.live_ex(u, v, x, p=1.0, mix=True)
        z = x ^ oracle.edge_hash(u, v)
        assert oracle.live_ex(u, v, x, p=0.3, mix=True) == (oracle.fmix32(z) < oracle.threshold(0.3))


def _arc_weights(xadj, adj, fn):
    n = xadj.shape[0] - 1
    src = np.repeat(np.arange(n), np.diff(xadj))
    lo, hi = np.minimum(src, adj), np.maximum(src, adj)
    return fn(lo, hi)


def test_uniform_weights_equal_uniform_p():
    xadj, adj = synth.chung_lu(800, 3200, 2.3, 31)
    for p in (0.01, 0.1, 0.5):
        w = _arc_weights(xadj, adj, lambda lo, hi: np.full(lo.shape, p))
        a = oracle.select_seeds(xadj, adj, 12, 64, p, 5)
        b = oracle.select_seeds_ex(xadj, adj, 12, 64, 0.0, 5, weights=w)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(oracle.labels(xadj, adj, 64, p, 5)[0],
                              oracle.labels_ex(xadj, adj, 64, 0.9, 5, weights=w)[0])


def test_zero_one_weights_give_the_components_of_the_certain_edges():
    xadj, adj = synth.random_graph(300, 700, 32)
    n = 300
    keep = lambda lo, hi: ((lo * 7 + hi * 13) % 3 == 0)  # noqa: E731
    w = _arc_weights(xadj, adj, lambda lo, hi: keep(lo, hi).astype(np.float64))
    src = np.repeat(np.arange(n), np.diff(xadj))
    sel = keep(np.minimum(src, adj), np.maximum(src, adj))
    A = coo_matrix((np.ones(int(sel.sum())), (src[sel], adj[sel])), shape=(n, n))
    _, comp = connected_components(A, directed=False)
    minid = np.full(comp.max() + 1, n)
    np.minimum.at(minid, comp, np.arange(n))
    lab, siz = oracle.labels_ex(xadj, adj, 16, 0.0, 9, weights=w)
    for r in range(16):
        assert np.array_equal(lab[:, r], minid[comp])
    for mix in (False, True):
        assert np.array_equal(oracle.labels_ex(xadj, adj, 4, 0.0, 9, weights=w, mix=mix)[0][:, 0],
                              minid[comp])


def test_weighted_and_mixed_live_rates_within_five_standard_errors():
    rng = np.random.default_rng(11)
    X = oracle.mt19937(1234, 40000)
    for (u, v, w, mix) in ((1, 2, 0.3, False), (5, 77, 0.05, False), (8, 9, 0.05, True),
                           (10, 400, 0.3, True)):
        hits = sum(oracle.live_ex(u, v, int(x), p=w, mix=mix) if mix else
                   oracle.live_ex(u, v, int(x), w=w) for x in X)
        q = oracle.edge_code(w) / 2.0 ** 32
        se = math.sqrt(q * (1 - q) / len(X))
        assert abs(hits / len(X) - q) < 5 * se, (u, v, w, mix)
    del rng


def test_mixed_hash_decorrelates_edges_the_plain_xor_never_samples_together():
    """With the plain XOR at p = 2^-6, an edge is live only when the top six
    bits of X_r equal those of its hash, so two edges whose hashes differ there
    are never live in the same sample; through fmix32 they are co-live at a
    rate near p^2."""
    p = 2.0 ** -6
    pairs = []
    for u in range(1, 200):
        h1, h2 = oracle.edge_hash(0, u), oracle.edge_hash(0, u + 1000)
        if (h1 >> 26) != (h2 >> 26):
            pairs.append((u, u + 1000))
        if len(pairs) == 3:
            break
    X = oracle.mt19937(99, 60000)
    for u, v in pairs:
        plain = sum(oracle.live(0, u, int(x), p) and oracle.live(0, v, int(x), p) for x in X)
        assert plain == 0
        mixed = sum(oracle.live_ex(0, u, int(x), p=p, mix=True)
                    and oracle.live_ex(0, v, int(x), p=p, mix=True) for x in X)
        se = math.sqrt(p * p * (1 - p * p) / len(X))
        assert abs(mixed / len(X) - p * p) < 5 * se


def test_options_greedy_agrees_with_its_tables_and_bfs_spread():
    xadj, adj = synth.chung_lu(600, 3000, 2.2, 33)
    w = _arc_weights(xadj, adj, lambda lo, hi: ((lo * 31 + hi * 17) % 100) / 1000.0)  # U-like [0, 0.1)
    for kw in (dict(weights=w), dict(mix=True), dict(weights=w, mix=True)):
        lab, siz = oracle.labels_ex(xadj, adj, 48, 0.05, 3, **kw)
        s, g = oracle.select_seeds_ex(xadj, adj, 10, 48, 0.05, 3, **kw)
        s2, g2 = oracle.greedy_from_tables(lab, siz, 10)
        assert np.array_equal(s, s2) and np.array_equal(g, g2)
        for k in (0, 4, 9):
            assert oracle.estimate_spread_ex(xadj, adj, s[:k + 1], 48, 0.05, 3, **kw) == int(g[k])


def test_weights_must_be_symmetric_and_in_range():
    xadj, adj = synth.random_graph(50, 100, 34)
    w = np.full(adj.shape[0], 0.2)
    w[0] = 0.3  # one arc differs from its reverse
    with pytest.raises(ValueError):
        oracle.select_seeds_ex(xadj, adj, 3, 8, 0.0, 1, weights=w)
    for bad in (-0.1, 1.5, np.nan):
        w = np.full(adj.shape[0], bad)
        with pytest.raises(ValueError):
            oracle.labels_ex(xadj, adj, 8, 0.0, 1, weights=w)
