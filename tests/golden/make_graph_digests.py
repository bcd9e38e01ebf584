"""Write graph_sha256.txt: the SHA-256 of every synthetic workload graph.

The digest covers the int32 little-endian bytes of xadj followed by adj, so a
change of the generators, of numpy's PCG64 stream or of the CSR layout on any
machine shows up as a mismatch. Run from the repository root:

    python tests/golden/make_graph_digests.py
"""
import hashlib
import os
import sys

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))
from paper_2008_03095_gb300 import synth  # noqa: E402


def digest(xadj, adj):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(xadj, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(adj, dtype="<i4").tobytes())
    return h.hexdigest()


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "graph_sha256.txt")
    lines = ["# workload n m max_degree sha256(xadj||adj, int32 LE)"]
    for name in synth.WORKLOADS:
        xadj, adj = synth.workload_graph(name)
        n, m = len(xadj) - 1, len(adj) // 2
        lines.append(f"{name} {n} {m} {int(np.diff(xadj).max())} {digest(xadj, adj)}")
        print(lines[-1], flush=True)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
