"""The synthetic workload graphs are reproducible: their SHA-256 digests
(written by tests/golden/make_graph_digests.py) match on every machine.
The 4M-vertex graph (about a minute to generate) is left to that script."""
import hashlib
import os

import numpy as np
import pytest

from paper_2008_03095_gb300 import synth

_GOLD = os.path.join(os.path.dirname(__file__), "golden", "graph_sha256.txt")


def _table():
    rows = {}
    with open(_GOLD) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, n, m, dmax, sha = line.split()
            rows[name] = (int(n), int(m), int(dmax), sha)
    return rows


def test_every_workload_has_a_digest():
    assert set(_table()) == set(synth.WORKLOADS)


@pytest.mark.parametrize("name", ["powerlaw_n2000", "powerlaw_n15233", "powerlaw_n37154",
                                  "clustered_n334863"])
def test_workload_graph_digest(name):
    n, m, dmax, sha = _table()[name]
    xadj, adj = synth.workload_graph(name)
    assert (len(xadj) - 1, len(adj) // 2, int(np.diff(xadj).max())) == (n, m, dmax)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(xadj, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(adj, dtype="<i4").tobytes())
    assert h.hexdigest() == sha
