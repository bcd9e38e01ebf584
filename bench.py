#!/usr/bin/env python
"""Benchmark of the fused-sampling influence-maximization hot path on one GB300.

Workload (default): undirected power-law graph n=15,233, m=58,891 (exponent
2.3, max degree ~350; NetHEP shape), R=1024 simulations, K=50 seeds,
p in {0.005, 0.01, 0.05}, X_r from MT19937(7). One step = for each p, select
K seeds (all phases of the hot path: lane randoms, fused hash-sample +
components, size memo, first gains, CELF) and estimate the spread of the
selected set. Units: sampled edge visits, 2m*R per query (every arc in every
simulation counted once); value = units / time in GTEPS x R.

Timing: CUDA events on the launching stream around each step; the L2 cache is
flushed (256 MiB write) between steps, outside the timed intervals; W warm-up
steps; K timed steps; max over ranks. `--impl reference` times the CPU oracle
on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "K-seed selection wall time + sampled edge-visits/s (GTEPS×R), % HBM peak"
UNIT = "GTEPS×R"
WORKLOAD = "powerlaw_n15233"
REF_R = 64  # lanes per query in a reference-arm (CPU oracle) step


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    return ap.parse_args()


# ------------------------------------------------------------------ helpers


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, device=None):
    """Largest per-rank value (a time) over the process group, or the value
    itself when no group of more than one rank is initialized. Works with
    nccl (device tensor) and gloo (host tensor) alike."""
    import torch
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds_max, world):
    """Whole-job rate: every rank processed units_per_rank (replicas, weak
    scaling) and the job ended with its slowest rank."""
    return world * units_per_rank / seconds_max / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ reference arm


def run_reference(args, xadj, adj, w):
    """The CPU oracle on a bounded sample of the workload (REF_R lanes per query)."""
    import oracle

    m = adj.shape[0] // 2
    ps = w["ps"]

    def step():
        for p in ps:
            seeds, sigma = oracle.select_seeds(xadj, adj, w["K"], REF_R, p, w["rng_seed"])
            oracle.estimate_spread(xadj, adj, seeds, REF_R, p, w["rng_seed"])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    units = len(ps) * 2 * m * REF_R * args.steps
    value = units / dt / 1e9
    sample = ("oracle select_seeds + estimate_spread, K=%d, %d lanes per query (of R=%d), p in %s"
              % (w["K"], REF_R, w["R"], list(ps)))
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(args.workload, xadj, adj, w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def workload_config(name, xadj, adj, w):
    deg = np.diff(xadj)
    return {"workload": "%s: undirected power-law graph n=%d m=%d (max degree %d), R=%d, K=%d, "
                        "p in %s, rng_seed %d" % (name, xadj.shape[0] - 1, adj.shape[0] // 2,
                                                  int(deg.max()), w["R"], w["K"], list(w["ps"]),
                                                  w["rng_seed"]),
            "n": int(xadj.shape[0] - 1), "m": int(adj.shape[0] // 2), "R": w["R"], "K": w["K"],
            "p": list(w["ps"]), "rng_seed": w["rng_seed"],
            "l2": "flushed between timed steps (256 MiB device write)"}


# ------------------------------------------------------------------ our arm


def algorithmic_bytes(phase, n, m_up, R, T):
    """Minimum bytes one launch of `phase` must move (see the kernel table)."""
    nR = n * R
    if phase == "prep":
        return 4 * nR + nR / 8  # label table init + covered bitmap clear
    if phase == "compress":
        return 4 * nR  # read every slot once
    if phase == "gains":
        return 4 * nR + 8 * n  # read every slot once, write n keys
    if phase == "union":
        live = m_up * R * (T / 2.0 ** 32)
        return 8 * m_up + 8 * live  # edge list + both endpoint slots per live arc-lane
    return None


def celf_algorithmic_bytes(n, R, evaluations, extractions, refreshes):
    """Minimum bytes of one lazy-greedy launch, from its work counters: each
    exact gain evaluation reads the candidate's R labels, the R root sizes and
    R covered bits; each prefix extraction scans the n keys; each refresh
    re-evaluates every vertex (labels, sizes, covered bits) and rewrites the
    keys."""
    per_eval = 4 * R + 4 * R + R / 8
    return (evaluations * per_eval + extractions * 8 * n
            + refreshes * (n * per_eval + 8 * n))


def run_ours(args, xadj, adj, w):
    import torch

    import paper_2008_03095_gb300 as im
    from paper_2008_03095_gb300 import build as lib_build

    rank, world, local_rank = dist_env()
    lib_build.build()
    im.lib()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = xadj.shape[0] - 1
    m = adj.shape[0] // 2
    R, K, ps, seed = w["R"], w["K"], list(w["ps"]), w["rng_seed"]
    stream = torch.cuda.current_stream()
    im.im_set_stream(stream)

    g = im.im_graph_create(xadj, adj)
    ws = im.im_workspace_create(g, R)
    d_seeds = torch.empty((len(ps), K), dtype=torch.int32, device=dev)
    d_sigma = torch.empty((len(ps), K), dtype=torch.int64, device=dev)
    d_spread = torch.empty((len(ps),), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # The queries of a step are independent: each runs on its own stream with
    # its own workspace, forked from and joined back to the launching stream.
    q_streams = [torch.cuda.Stream(device=dev) for _ in ps]
    q_ws = [ws] + [im.im_workspace_create(g, R) for _ in ps[1:]]

    def step():
        fork = torch.cuda.Event()
        fork.record(stream)
        joins = []
        for i, p in enumerate(ps):
            qs = q_streams[i]
            qs.wait_event(fork)
            im.im_set_stream(qs)
            im.im_select_seeds_async(g, q_ws[i], K, R, p, seed, d_seeds[i], d_sigma[i])
            im.im_estimate_spread_async(g, q_ws[i], d_seeds[i], K, R, p, seed, d_spread[i:i + 1])
            done = torch.cuda.Event()
            done.record(qs)
            joins.append(done)
        for done in joins:
            stream.wait_event(done)
        im.im_set_stream(stream)

    def step_serial():  # one stream, for the per-kernel event breakdown
        for i, p in enumerate(ps):
            im.im_select_seeds_async(g, ws, K, R, p, seed, d_seeds[i], d_sigma[i])
            im.im_estimate_spread_async(g, ws, d_seeds[i], K, R, p, seed, d_spread[i:i + 1])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for w_ in q_ws:
        im.im_workspace_status(w_)

    def timed_steps(nsteps, fn=step):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        for k in range(nsteps):
            flush.zero_()
            starts[k].record(stream)
            fn()
            ends[k].record(stream)
        torch.cuda.synchronize()
        return sum(s.elapsed_time(e) for s, e in zip(starts, ends))

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = im.im_kernel_launches()
    total_ms = timed_steps(args.steps)
    launches = im.im_kernel_launches() - launches0
    clock_info = clocks.stop()
    for w_ in q_ws:
        im.im_workspace_status(w_)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dev)
        torch.distributed.barrier()

    seeds_h = d_seeds.cpu().numpy()
    sigma_h = d_sigma.cpu().numpy().astype(np.uint64)
    spread_h = d_spread.cpu().numpy().astype(np.uint64)
    consistent = bool(all(int(spread_h[i]) == int(sigma_h[i, -1]) for i in range(len(ps))))

    # Per-kernel times: the same steps again with events around every launch,
    # then each p on its own (kernel times and device work counters per query).
    im.im_workspace_stats(ws)
    im.im_profile_enable(True)
    serial_ms = timed_steps(args.steps, step_serial)
    prof = im.im_profile_read()
    by_p = {}
    for i, p in enumerate(ps):
        im.im_profile_read()
        im.im_workspace_stats(ws)
        for _ in range(args.steps):
            flush.zero_()
            im.im_select_seeds_async(g, ws, K, R, p, seed, d_seeds[i], d_sigma[i])
            im.im_estimate_spread_async(g, ws, d_seeds[i], K, R, p, seed, d_spread[i:i + 1])
        pp = im.im_profile_read()
        st = im.im_workspace_stats(ws)
        by_p[str(p)] = {"avg_us": {k: round(v[0] / v[1] * 1e3, 2) for k, v in pp.items() if v[1]},
                        "per_query": {k: v / args.steps for k, v in st.items()}}
    im.im_profile_enable(False)

    units_per_step = len(ps) * 2 * m * R
    value = job_throughput(units_per_step * args.steps, total_ms / 1e3, world)
    per_kernel = {k: {"total_ms": v[0], "launches": v[1],
                      "avg_us": (v[0] / v[1] * 1e3) if v[1] else None} for k, v in prof.items()}
    peak, peak_kind = measured_peaks()
    T = {p: im.im_sampling_threshold(p) for p in ps}
    dominant = max(prof, key=lambda k: prof[k][0])
    roof = None
    bytes_per_launch = None
    if dominant in ("prep", "compress", "gains"):
        bytes_per_launch = algorithmic_bytes(dominant, n, 0, R, 0)
    elif dominant == "union":
        bytes_per_launch = statistics.mean(algorithmic_bytes("union", n, g_m_up(xadj, adj), R, T[p])
                                           for p in ps)
    note = None
    if dominant == "celf":
        # per-launch average over the queries of a step, from the device counters
        q = [by_p[str(p)]["per_query"] for p in ps]
        bytes_per_launch = statistics.mean(
            celf_algorithmic_bytes(n, R, x["celf_evaluations"], x["celf_extractions"],
                                   x["celf_refreshes"]) for x in q)
        note = ("latency-bound: one block runs the sequential lazy-greedy rounds while the "
                "grid waits; the HBM roof is reported for its algorithmic bytes")
    if bytes_per_launch is not None:
        avg_s = prof[dominant][0] / prof[dominant][1] / 1e3
        achieved = bytes_per_launch / avg_s / 1e9
        roof = {"kernel": "k_" + dominant, "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": committed_traffic("k_" + dominant, args.workload),
                "bytes_per_launch": bytes_per_launch}
        if note:
            roof["note"] = note
    else:
        roof = {"kernel": "k_" + dominant, "bound": "latency", "achieved": None, "peak": peak,
                "unit": "GB/s", "frac": None, "peak_kind": peak_kind, "traffic": None}
    # the best HBM-bound kernel, reported beside the dominant one
    hbm = {}
    for ph in ("prep", "compress", "gains"):
        if prof[ph][1]:
            b = algorithmic_bytes(ph, n, 0, R, 0)
            a = b / (prof[ph][0] / prof[ph][1] / 1e3) / 1e9
            hbm["k_" + ph] = {"achieved_gbs": a, "frac": a / peak, "bytes_per_launch": b}

    # The component pipeline (label init, fused sample + union, size memo,
    # first gains) against its algorithmic floor 8m + 20nR bytes per query:
    # the CSR once, labels written, read for sizes, sizes written, labels and
    # sizes read for the first gains.
    cc_phases = ("prep", "union", "compress", "gains")
    cc_us = sum(prof[ph][0] / prof[ph][1] * 1e3 for ph in cc_phases if prof[ph][1])
    cc_bytes = 8 * m + 4 * (n + 1) + 20 * n * R
    cc_gbs = cc_bytes / (cc_us / 1e6) / 1e9
    cc = {"phases": list(cc_phases), "us_per_query": cc_us, "bytes_per_query": cc_bytes,
          "achieved_gbs": cc_gbs, "frac": cc_gbs / peak, "peak": peak, "peak_kind": peak_kind}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(args.workload, xadj, adj, w),
        "select_plus_spread_ms_per_query": total_ms / args.steps / len(ps),
        "queries_concurrent": len(ps),
        "ms_per_step_one_stream": serial_ms / args.steps,
        "gpu_launches": int(launches), "roofline": roof, "hbm_kernels": hbm,
        "component_pipeline": cc,
        "per_kernel": per_kernel, "per_p": by_p, "clocks": clock_info, "consistent_spread": consistent,
        "paper_context": "NetHEP (15,235 v / 58,892 e), K=50, p=0.01: 0.08 s on 2x Xeon "
                         "E5-2620v4, 16 threads (Table 4); R not stated",
    }
    out["_gpu_results"] = (seeds_h, sigma_h, spread_h)
    out["_e2e"] = lambda: run_e2e(args, xadj, adj, w, im, torch)
    for w_ in q_ws:
        w_.close()
    g.close()
    return out


def g_m_up(xadj, adj):
    n = xadj.shape[0] - 1
    src = np.repeat(np.arange(n), np.diff(xadj))
    return int(np.count_nonzero(adj > src))


def committed_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary (profiles/dram_traffic.txt)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel \
                    and parts[1] == workload:
                return float(parts[2])
    return None


def run_e2e(args, xadj, adj, w, im, torch):
    """Same metric through the blocking C ABI with host buffers: graph upload
    from pinned host memory, select (host outputs), spread (host seeds), free."""
    n = xadj.shape[0] - 1
    m = adj.shape[0] // 2
    R, K, ps, seed = w["R"], w["K"], list(w["ps"]), w["rng_seed"]
    hx = torch.from_numpy(xadj).pin_memory()
    ha = torch.from_numpy(adj).pin_memory()
    seeds_buf = np.empty(K, dtype=np.int32)
    sigma_buf = np.empty(K, dtype=np.uint64)
    im.im_set_stream(None)

    def step():
        g = im.im_graph_create_raw(n, m, hx.data_ptr(), ha.data_ptr())
        for p in ps:
            im.im_select_seeds(g, K, R, p, seed, seeds_buf, sigma_buf)
            im.im_estimate_spread(g, seeds_buf, R, p, seed)
        g.close()

    step()
    torch.cuda.synchronize()
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        step()
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, torch.device("cuda", torch.cuda.current_device()))
    world = torch.distributed.get_world_size() if torch.distributed.is_initialized() else 1
    units = len(ps) * 2 * m * R * args.e2e_steps
    h2d = 4 * (n + 1) + 8 * m + len(ps) * K * 4
    d2h = len(ps) * (K * 4 + K * 8 + 8)
    return {"value": job_throughput(units, dt, world), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
            "ms_per_step": dt * 1e3 / args.e2e_steps,
            "path": "im_graph_create (pinned host CSR) + im_select_seeds + im_estimate_spread "
                    "per p + im_graph_destroy"}


def run_cpu_baseline(xadj, adj, w, gpu_results):
    """The oracle, as it stands, single-threaded, on one full step of the workload."""
    import oracle

    m = adj.shape[0] // 2
    R, K, ps, seed = w["R"], w["K"], list(w["ps"]), w["rng_seed"]
    seeds_g, sigma_g, spread_g = gpu_results
    parity = True
    t0 = time.perf_counter()
    for i, p in enumerate(ps):
        s, sg = oracle.select_seeds(xadj, adj, K, R, p, seed)
        sp = oracle.estimate_spread(xadj, adj, s, R, p, seed)
        parity &= bool(np.array_equal(s, seeds_g[i]) and np.array_equal(sg, sigma_g[i])
                       and sp == int(spread_g[i]))
    dt = time.perf_counter() - t0
    return {"value": len(ps) * 2 * m * R / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one full step (select K=%d + spread, R=%d, p in %s), single thread"
                      % (K, R, ps), "seconds": dt, "cpu": cpu_model()}, parity


def main():
    args = parse_args()
    rank, world, local_rank = dist_env()
    from paper_2008_03095_gb300 import synth

    w = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        if rank != 0:
            return 0
        xadj, adj = synth.workload_graph(args.workload)
        print(json.dumps(run_reference(args, xadj, adj, w)))
        return 0

    import torch

    if world > 1:
        import datetime
        torch.distributed.init_process_group(
            backend="nccl" if torch.cuda.is_available() else "gloo",
            timeout=datetime.timedelta(minutes=10))
    xadj, adj = synth.workload_graph(args.workload)
    out = run_ours(args, xadj, adj, w)
    gpu_results = out.pop("_gpu_results")
    e2e_fn = out.pop("_e2e")
    out["e2e"] = e2e_fn()
    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            cb, parity = run_cpu_baseline(xadj, adj, w, gpu_results)
            out["cpu_baseline"] = cb
            out["parity_vs_oracle"] = parity
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
