"""Write oracle_expected_seeds.txt: the oracle's seed sequence and sigma*R for
the workloads too large for the oracle to run inside the test suite.

Only oracle/ computes anything here (its OpenMP build, which returns the same
results as the single-threaded one: every greedy step is the maximum gain with
the lowest id among equal gains). The graphs come from the seeded generators,
and each line records the graph's SHA-256 so that a test can tell a changed
graph from a wrong selection. Run from the repository root (about 10 minutes
and 20 GB of host memory on 8 cores for the 4M-vertex graph):

    python tests/golden/make_oracle_expected.py [workload ...]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), "..", ".."))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import oracle  # noqa: E402
from make_graph_digests import digest  # noqa: E402
from paper_2008_03095_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_expected_seeds.txt")
WORKLOADS = ("clustered_n334863", "powerlaw_n4m")
HEADER = ("# workload p K R rng_seed graph_sha256 | seeds s_1..s_K | sigmaR_1..sigmaR_K\n"
          "# written by tests/golden/make_oracle_expected.py (oracle/ only)")


def read_expected(path=OUT):
    """{(workload, p): (sha256, K, R, rng_seed, seeds int32[K], sigma uint64[K])}"""
    out = {}
    if not os.path.exists(path):
        return out
    with open(path) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            head, seeds, sigma = line.split("|")
            name, p, K, R, seed, sha = head.split()
            out[(name, float(p))] = (sha, int(K), int(R), int(seed),
                                     np.array(seeds.split(), dtype=np.int32),
                                     np.array(sigma.split(), dtype=np.uint64))
    return out


def main(names):
    oracle.use_all_cores(True)
    rows = {k: v for k, v in read_expected().items() if k[0] not in names}
    lines = {}
    for (name, p), (sha, K, R, seed, s, g) in rows.items():
        lines[(name, p)] = "%s %r %d %d %d %s | %s | %s" % (
            name, p, K, R, seed, sha, " ".join(map(str, s)), " ".join(map(str, g)))
    for name in names:
        w = synth.WORKLOADS[name]
        xadj, adj = synth.workload_graph(name)
        sha = digest(xadj, adj)
        for p in w["ps"]:
            t0 = time.time()
            seeds, sigma = oracle.select_seeds(xadj, adj, w["K"], w["R"], p, w["rng_seed"])
            print("%s p=%g: %.0f s on %d threads, sigmaR[K-1]=%d" % (
                name, p, time.time() - t0, oracle.threads(), int(sigma[-1])), flush=True)
            lines[(name, p)] = "%s %r %d %d %d %s | %s | %s" % (
                name, p, w["K"], w["R"], w["rng_seed"], sha, " ".join(map(str, seeds)),
                " ".join(map(str, sigma)))
    with open(OUT, "w") as f:
        f.write(HEADER + "\n" + "\n".join(lines[k] for k in sorted(lines)) + "\n")


if __name__ == "__main__":
    main(tuple(sys.argv[1:]) or WORKLOADS)
