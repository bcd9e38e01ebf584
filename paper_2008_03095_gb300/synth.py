"""Seeded synthetic undirected graphs shaped like the paper's networks.

This module only builds inputs (CSR arrays); it holds none of the method's
arithmetic. Every generator is deterministic in its seed (numpy PCG64), emits a
simple graph (no self-loops, no duplicate edges), permutes vertex ids with the
same stream so that id is uncorrelated with degree, and returns a symmetric CSR
(int32 `xadj[n+1]`, int32 `adj[2m]`) with every neighbour list sorted.

The paper's datasets (Table 3: NetHEP, NetPhy, Amazon, ...) are not available;
these generators stand in for them with the same vertex/edge counts and degree
shapes.
"""
import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def csr_from_edges(n, u, v):
    """Symmetric CSR from an undirected edge list (u[i], v[i]), lists sorted."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    order = np.argsort(src * n + dst, kind="stable")
    adj = dst[order].astype(np.int32)
    deg = np.bincount(src, minlength=n)
    xadj = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=xadj[1:])
    if xadj[-1] >= 2 ** 31:
        raise ValueError("graph too large for int32 CSR")
    return xadj.astype(np.int32), adj


def _draw_unique_edges(rng, n, m, prob, forbidden=None):
    """First m distinct non-loop pairs, in draw order, endpoints drawn ∝ prob."""
    cdf = np.cumsum(prob, dtype=np.float64)
    cdf /= cdf[-1]
    collected = np.empty(0, dtype=np.int64)
    got = 0
    while True:
        batch = int((m - got) * 1.25) + 1024
        a = np.minimum(np.searchsorted(cdf, rng.random(batch), side="right"), n - 1)
        b = np.minimum(np.searchsorted(cdf, rng.random(batch), side="right"), n - 1)
        keep = a != b
        lo = np.minimum(a[keep], b[keep]).astype(np.int64)
        hi = np.maximum(a[keep], b[keep]).astype(np.int64)
        collected = np.concatenate([collected, lo * n + hi])
        uniq, first = np.unique(collected, return_index=True)
        if forbidden is not None and forbidden.size:
            ok = ~np.isin(uniq, forbidden, assume_unique=False)
            uniq, first = uniq[ok], first[ok]
        got = uniq.shape[0]
        if got >= m:
            keys = uniq[np.argsort(first, kind="stable")[:m]]
            return keys // n, keys % n


def _finish(rng, n, lo, hi):
    perm = rng.permutation(n).astype(np.int64)
    return csr_from_edges(n, perm[lo], perm[hi])


def chung_lu_weights(n, m, gamma, dmax=None):
    """w_i = (i + i0)^(-1/(gamma-1)) scaled to sum 2m; i0 chosen so max w ≈ dmax."""
    alpha = 1.0 / (gamma - 1.0)
    idx = np.arange(n, dtype=np.float64)

    def weights(i0):
        w = (idx + i0) ** -alpha
        return w * (2.0 * m / w.sum())

    i0 = 1.0
    if dmax is not None and weights(1.0)[0] > dmax:
        lo, hi = 1.0, float(n)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if weights(mid)[0] > dmax:
                lo = mid
            else:
                hi = mid
        i0 = hi
    return weights(i0)


def chung_lu(n, m, gamma, seed, dmax=None):
    """Power-law Chung-Lu graph with exactly m distinct undirected edges."""
    rng = _rng(seed)
    w = chung_lu_weights(n, m, gamma, dmax)
    lo, hi = _draw_unique_edges(rng, n, m, w)
    return _finish(rng, n, lo, hi)


def clustered(n, m, seed, clique_frac=0.5, kmin=4, kmax=8, geo_p=0.25, n_hubs=24,
              hub_deg=(400, 550)):
    """Low-skew clustered graph (co-purchase shape).

    About `clique_frac` of the vertices are split into disjoint cliques of size
    U{kmin..kmax} (all clique edges present); the remaining edges are drawn
    Chung-Lu style with geometric-tailed weights 1 + Geom (mean 1/geo_p) plus
    `n_hubs` hubs whose expected degree is U[hub_deg], until exactly m edges.
    """
    rng = _rng(seed)
    members = rng.permutation(n)
    target = int(clique_frac * n)
    sizes = []
    tot = 0
    while tot < target:
        s = int(rng.integers(kmin, kmax + 1))
        if tot + s > n:
            break
        sizes.append(s)
        tot += s
    lo_l, hi_l = [], []
    pos = 0
    for s in sizes:
        c = np.sort(members[pos:pos + s])
        pos += s
        iu, ju = np.triu_indices(s, 1)
        lo_l.append(c[iu])
        hi_l.append(c[ju])
    clo = np.concatenate(lo_l).astype(np.int64)
    chi = np.concatenate(hi_l).astype(np.int64)
    if clo.shape[0] > m:
        raise ValueError("cliques alone exceed m")
    m_rest = m - clo.shape[0]
    w = rng.geometric(geo_p, size=n).astype(np.float64)
    hubs = rng.choice(n, size=n_hubs, replace=False)
    hub_w = rng.uniform(hub_deg[0], hub_deg[1], size=n_hubs)
    w[hubs] = 0.0
    w *= (2.0 * m_rest - hub_w.sum()) / w.sum()
    w[hubs] = hub_w
    forbidden = clo * n + chi
    lo, hi = _draw_unique_edges(rng, n, m_rest, w, forbidden=forbidden)
    return _finish(rng, n, np.concatenate([clo, lo]), np.concatenate([chi, hi]))


def random_graph(n, m, seed):
    """Uniform simple graph G(n, m) (for small test cases)."""
    rng = _rng(seed)
    m = min(m, n * (n - 1) // 2)
    if m == 0:
        return np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32)
    lo, hi = _draw_unique_edges(rng, n, m, np.ones(n))
    return _finish(rng, n, lo, hi)


def edge_weights(xadj, adj, kind, seed):
    """One probability per CSR arc, equal on both arcs of an edge, drawn per
    undirected edge (numpy PCG64) as in the paper's weight settings (Section
    4): "uniform" U[0, 0.1] or "normal" N(0.05, 0.025) clipped to [0, 1]."""
    n = xadj.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(xadj))
    dst = adj.astype(np.int64)
    key = np.minimum(src, dst) * n + np.maximum(src, dst)
    uniq, inv = np.unique(key, return_inverse=True)
    rng = _rng(seed)
    if kind == "uniform":
        vals = rng.uniform(0.0, 0.1, size=uniq.shape[0])
    elif kind == "normal":
        vals = np.clip(rng.normal(0.05, 0.025, size=uniq.shape[0]), 0.0, 1.0)
    else:
        raise ValueError("unknown weight setting %r" % kind)
    return vals[inv].astype(np.float64)


def batched_instances(count=256, seed=40, n_range=(500, 200_000), Rs=(256, 1024, 2048),
                      K_range=(5, 100), p_range=(0.001, 0.1)):
    """Uneven independent instances for a batched launch: per instance a
    Chung-Lu graph with n log-uniform in n_range, m/n ~ U[2, 15], exponent
    ~ U[2, 3] and generator seed 1000 + i, and a query with p log-uniform in
    p_range, R drawn from Rs, K ~ U{K_range} (at most n) and rng_seed 7 + i.
    Parameters come from PCG64(seed); graphs are built lazily by `graph()`."""
    rng = _rng(seed)
    out = []
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    plo, phi = np.log(p_range[0]), np.log(p_range[1])
    for i in range(count):
        n = int(round(np.exp(rng.uniform(lo, hi))))
        ratio = rng.uniform(2.0, 15.0)
        m = min(int(round(n * ratio)), n * (n - 1) // 2)
        gamma = rng.uniform(2.0, 3.0)
        p = float(np.exp(rng.uniform(plo, phi)))
        R = int(Rs[int(rng.integers(0, len(Rs)))])
        K = int(min(rng.integers(K_range[0], K_range[1] + 1), n))
        out.append(dict(n=n, m=m, gamma=gamma, graph_seed=1000 + i, p=p, R=R, K=K,
                        rng_seed=7 + i))
    return out


def instance_graph(inst):
    return chung_lu(inst["n"], inst["m"], inst["gamma"], inst["graph_seed"])


# Workload recipes: graph builder, its arguments, and the query parameters.
WORKLOADS = {
    # n=2,000 m=8,000 power-law (exponent 2.5)
    "powerlaw_n2000": dict(gen=chung_lu, args=(2000, 8000, 2.5, 1), kw={}, R=256, K=10,
                           ps=(0.01,), rng_seed=7),
    # n=15,233 m=58,891 power-law (exponent 2.3, max degree ~350): NetHEP shape
    "powerlaw_n15233": dict(gen=chung_lu, args=(15233, 58891, 2.3, 2), kw=dict(dmax=350.0),
                            R=1024, K=50, ps=(0.005, 0.01, 0.05), rng_seed=7),
    # n=37,154 m=231,584 power-law (exponent 2.1): NetPhy shape
    "powerlaw_n37154": dict(gen=chung_lu, args=(37154, 231584, 2.1, 3), kw={}, R=2048, K=50,
                            ps=(0.01, 0.05), rng_seed=7),
    # n=334,863 m=925,872 clustered low-skew: co-purchase (Amazon) shape
    "clustered_n334863": dict(gen=clustered, args=(334863, 925872, 4), kw={}, R=2048, K=50,
                              ps=(0.01, 0.05), rng_seed=7),
    # n=4,000,000 m=35,000,000 power-law (exponent 2.2)
    "powerlaw_n4m": dict(gen=chung_lu, args=(4_000_000, 35_000_000, 2.2, 41), kw={}, R=512,
                         K=50, ps=(0.01,), rng_seed=7),
}


def workload_graph(name):
    w = WORKLOADS[name]
    return w["gen"](*w["args"], **w["kw"])
