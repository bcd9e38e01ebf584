"""Shared helpers for the tests: golden-file parsing, explicit live masks and
small independent reference computations (plain Python / scipy)."""
import os
from collections import deque

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def worked_example():
    """Graph, per-arc live mask and expected values of the Figures 3-4 example."""
    from paper_2008_03095_gb300.synth import csr_from_edges
    rec = {row[0]: row[1:] for row in golden_lines("worked_example_fig3_fig4.txt")}
    ids = {c: i for i, c in enumerate("ABCDE")}

    def pairs(tokens):
        return [tuple(sorted((ids[t[0]], ids[t[2]]))) for t in tokens]

    edges = pairs(rec["edges"])
    xadj, adj = csr_from_edges(5, [e[0] for e in edges], [e[1] for e in edges])
    live = [set(pairs(rec["live1"])), set(pairs(rec["live2"]))]
    mask = arc_mask(xadj, adj, lambda u, v, r: tuple(sorted((u, v))) in live[r], 2)
    exp = dict(labels=np.array([[int(x) for x in rec["labels1"]], [int(x) for x in rec["labels2"]]]).T,
               mg=[int(x) for x in rec["mg"]], first_seed=int(rec["first_seed"][0]),
               first_sigmaR=int(rec["first_sigmaR"][0]))
    return xadj, adj, mask, exp


def arc_mask(xadj, adj, pred, R):
    """uint8 [2m, R] with mask[a, r] = pred(u, v, r) for arc a = (u, v)."""
    n = xadj.shape[0] - 1
    mask = np.zeros((adj.shape[0], R), dtype=np.uint8)
    for u in range(n):
        for a in range(xadj[u], xadj[u + 1]):
            for r in range(R):
                mask[a, r] = 1 if pred(u, int(adj[a]), r) else 0
    return mask


def edge_list(xadj, adj):
    n = xadj.shape[0] - 1
    out = []
    for u in range(n):
        for a in range(xadj[u], xadj[u + 1]):
            v = int(adj[a])
            if u < v:
                out.append((u, v))
    return out


def py_reach(n, live_edges, seeds):
    """Vertices reachable from `seeds` over undirected `live_edges` (plain BFS)."""
    nbr = [[] for _ in range(n)]
    for u, v in live_edges:
        nbr[u].append(v)
        nbr[v].append(u)
    seen = set(int(s) for s in seeds)
    q = deque(seen)
    while q:
        u = q.popleft()
        for v in nbr[u]:
            if v not in seen:
                seen.add(v)
                q.append(v)
    return seen


def uf_min_labels(n, live_edges):
    """Union-find with path halving; label = minimum id in the component."""
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for u, v in live_edges:
        a, b = find(u), find(v)
        if a != b:
            parent[max(a, b)] = min(a, b)
    return np.array([find(v) for v in range(n)], dtype=np.int64)
