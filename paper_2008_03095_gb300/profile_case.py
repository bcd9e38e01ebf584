"""Run the bandwidth kernels of one workload query for a profiler, without the
lazy greedy: the component pipeline up to the first-seed gains (k_prep,
k_union, k_compress, k_gains through im_debug_first_gains) and the spread of
a fixed seed set (k_prep, k_spread through im_estimate_spread; after a
hand-over also k_union, k_spread_mark and k_spread_count), each `--repeat`
times on one resident graph.

    python -m paper_2008_03095_gb300.profile_case --workload powerlaw_n37154 --p 0.05

The seed set of the spread is the K highest-degree vertices (lowest id first
on equal degree), or with `--selected-seeds` the seeds that im_select_seeds
picks (selected once, before the profiled runs). `--select` profiles whole
selections instead (the lazy greedy included); `--ext-refresh 1|2` forces the
lazy greedy's bulk refresh into a launch of its own or inside the launch.
Prints one JSON line with the per-phase event times.
"""
import argparse
import json
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="powerlaw_n37154")
    ap.add_argument("--p", type=float, default=None)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--no-spread", action="store_true")
    ap.add_argument("--spread-only", action="store_true",
                    help="run only the spread, from an async workspace")
    ap.add_argument("--chung-lu", default=None,
                    help="n,m,gamma,seed: a Chung-Lu graph instead of a named workload")
    ap.add_argument("--R", type=int, default=None)
    ap.add_argument("--selected-seeds", action="store_true",
                    help="spread the seeds im_select_seeds picks instead of the top-degree ones")
    ap.add_argument("--select", action="store_true", help="profile whole selections")
    ap.add_argument("--ext-refresh", type=int, default=0,
                    help="1: the bulk refresh as a launch of its own; 2: inside the launch")
    args = ap.parse_args(argv)

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_2008_03095_gb300 as im
    from paper_2008_03095_gb300 import build, synth

    build.build()
    if args.chung_lu:
        n_, m_, gamma_, gseed = args.chung_lu.split(",")
        xadj, adj = synth.chung_lu(int(n_), int(m_), float(gamma_), int(gseed))
        w = dict(R=512, K=50, rng_seed=7, ps=(0.01,))
        args.workload = "chung_lu(%s)" % args.chung_lu
    else:
        w = synth.WORKLOADS[args.workload]
        xadj, adj = synth.workload_graph(args.workload)
    p = w["ps"][-1] if args.p is None else args.p
    R = w["R"] if args.R is None else args.R
    K, seed = w["K"], w["rng_seed"]
    deg = np.diff(xadj)
    seeds = np.argsort(-deg, kind="stable")[:K].astype(np.int32)
    torch.cuda.set_device(0)
    g = im.im_graph_create(xadj, adj)
    if args.ext_refresh:
        im.im_debug_override(im.IM_OVR_CELF_EXT_REFRESH, args.ext_refresh)
    if args.selected_seeds:
        seeds, _ = im.im_select_seeds(g, K, R, p, seed)
        seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    mg = np.zeros(1, dtype=np.uint64)
    if args.spread_only:
        ws = im.im_workspace_create(g, R)
        d_seeds = torch.from_numpy(seeds).cuda()
        d_sigma = torch.empty(1, dtype=torch.int64, device="cuda")
        im.im_set_stream(torch.cuda.current_stream())
    im.im_profile_enable(True)
    for _ in range(args.repeat):
        if args.spread_only:
            im.im_estimate_spread_async(g, ws, d_seeds, K, R, p, seed, d_sigma)
            continue
        if args.select:
            im.im_select_seeds(g, K, R, p, seed)
            continue
        mg = im.im_debug_first_gains(g, R, p, seed)
        if not args.no_spread:
            im.im_estimate_spread(g, seeds, R, p, seed)
    prof = im.im_profile_read()
    im.im_profile_enable(False)
    if args.spread_only:
        im.im_workspace_status(ws)
        ws.close()
        im.im_set_stream(None)
    g.close()
    print(json.dumps({"workload": args.workload, "p": p, "R": R, "repeat": args.repeat,
                      "max_first_gain": int(mg.max()),
                      "avg_us": {k: round(v[0] / v[1] * 1e3, 2) for k, v in prof.items() if v[1]}}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
