#!/usr/bin/env python
"""Benchmark of the fused-sampling influence-maximization hot path on one GB300.

Workload (default, the largest single-GPU configuration): undirected
power-law Chung-Lu graph n=4,000,000, m=35,000,000 (exponent 2.2), R=512
simulations, K=50 seeds, p=0.01, X_r from MT19937(7). One step = select K
seeds (every phase of the hot path: lane randoms, fused hash-sample +
components, size memo, first gains, lazy greedy) and estimate the spread of
the selected set. Units: sampled edge visits, 2m*R per query (every arc in
every simulation counted once); value = units / time in GTEPS x R. The
label table (8.2 GB) is far larger than L2, so no flush is needed between
steps; a 256 MiB write flushes it anyway.

Timing: CUDA events on the launching stream around each step; W warm-up
steps; K timed steps; max over ranks. Two more workloads are measured the same
way with fewer steps and reported under `extra_workloads`. `--impl reference`
times the CPU oracle on a bounded sample of the same workload instead.
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
WORKLOAD = "powerlaw_n4m"
EXTRA_WORKLOADS = ("clustered_n334863", "powerlaw_n15233")
# Simulations of one oracle step: the reference arm (every timed step) and the
# CPU baseline (one step per build), a prefix X_0..X_{r-1} of the workload's R.
REF_LANES = {"powerlaw_n4m": 1, "clustered_n334863": 8, "powerlaw_n37154": 16,
             "powerlaw_n15233": 64, "powerlaw_n2000": 256}
CPU_LANES = {"powerlaw_n4m": (2, 16), "clustered_n334863": (32, 256),
             "powerlaw_n37154": (64, 512), "powerlaw_n15233": (256, 1024),
             "powerlaw_n2000": (256, 256)}  # (single thread, all cores)
# Workloads whose oracle step is select_seeds alone: every oracle call first
# validates the CSR (about 10 s at 70M arcs), so select + spread would double
# the step; leaving out the spread only makes the oracle's rate look better.
ORACLE_SELECT_ONLY = ("powerlaw_n4m",)
FLUSH_BYTES = 256 << 20


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--extra-steps", type=int, default=5)
    ap.add_argument("--batch", type=int, default=256,
                    help="queries of the batched-launch leg (0: skip it)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--serve", type=int, default=1000,
                    help="queries per offered load of the serving leg (0: skip it)")
    ap.add_argument("--serve-rates", default="50,200,1000")
    return ap.parse_args(argv)


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
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def workload_config(name, xadj, adj, w, R=None, note=None):
    deg = np.diff(xadj)
    R = w["R"] if R is None else R
    shape = "clustered low-skew" if name.startswith("clustered") else "power-law"
    cfg = {"workload": "%s: undirected %s graph n=%d m=%d (max degree %d), R=%d, K=%d, "
                       "p in %s, rng_seed %d" % (name, shape, xadj.shape[0] - 1,
                                                 adj.shape[0] // 2, int(deg.max()), R, w["K"],
                                                 list(w["ps"]), w["rng_seed"]),
           "n": int(xadj.shape[0] - 1), "m": int(adj.shape[0] // 2), "R": R, "K": w["K"],
           "p": list(w["ps"]), "rng_seed": w["rng_seed"],
           "l2": "label table larger than L2 (n*R*4 bytes); a 256 MiB device write also "
                 "flushes L2 between timed steps"}
    if note:
        cfg["note"] = note
    return cfg


def stored_oracle(name):
    """{p: (seeds, sigma)} written by tests/golden/make_oracle_expected.py."""
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    try:
        from make_oracle_expected import read_expected
    except Exception:
        return {}
    return {p: (v[4], v[5]) for (n, p), v in read_expected().items() if n == name}


# ------------------------------------------------------------------ reference arm


def oracle_step(oracle, xadj, adj, w, lanes, spread=True):
    for p in w["ps"]:
        seeds, sigma = oracle.select_seeds(xadj, adj, w["K"], lanes, p, w["rng_seed"])
        if spread:
            oracle.estimate_spread(xadj, adj, seeds, lanes, p, w["rng_seed"])


def oracle_step_kind(name):
    return ("select_seeds" if name in ORACLE_SELECT_ONLY
            else "select_seeds + estimate_spread")


def run_reference(args, xadj, adj, w):
    """The CPU oracle, single-threaded as it stands, on a bounded sample of
    the workload: every step selects K seeds and estimates their spread on
    the first REF_LANES simulations of the workload's R."""
    import oracle

    m = adj.shape[0] // 2
    lanes = REF_LANES.get(args.workload, 8)
    spread = args.workload not in ORACLE_SELECT_ONLY
    for _ in range(args.warmup):
        oracle_step(oracle, xadj, adj, w, lanes, spread)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(oracle, xadj, adj, w, lanes, spread)
    dt = time.perf_counter() - t0
    units = len(w["ps"]) * 2 * m * lanes * args.steps
    value = units / dt / 1e9
    sample = ("oracle %s, K=%d, the first %d of the workload's R=%d simulations, p in %s, "
              "per step" % (oracle_step_kind(args.workload), w["K"], lanes, w["R"],
                            list(w["ps"])))
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(args.workload, xadj, adj, w, R=lanes,
                                  note="R=%d sampled of the workload's %d; the metric is per "
                                       "sampled edge visit, so it compares across R"
                                       % (lanes, w["R"])),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------------ our arm


# Kernel of a profiling phase whose name differs from the phase's.
KERNEL_OF_PHASE = {"spread_cc": "k_spread_count", "spread_mark": "k_spread_mark"}


def algorithmic_bytes(phase, n, m_up, R, T):
    """Minimum bytes one launch of `phase` must move (see the kernel table)."""
    nR = n * R
    if phase == "prep":
        return 4 * nR + nR / 8  # label table init + covered bitmap clear
    if phase == "compress":
        return 4 * nR  # read every slot once
    if phase == "gains":
        return 4 * nR + 8 * n  # read every slot once, write n keys
    if phase == "spread_cc":
        return 4 * nR + nR / 8  # the spread's count: every slot once, its own mark bit
    if phase == "union":
        live = m_up * R * (T / 2.0 ** 32)
        return 8 * m_up + 8 * live  # edge list + both endpoint slots per live arc-lane
    return None


def celf_method_bytes(n, R, evaluations, extractions):
    """Bytes the method itself moves in one lazy-greedy launch (the marginal-
    gain reduce of Algorithm 7): each exact evaluation reads the candidate's R
    labels, the R root sizes and R covered bits; each prefix extraction scans
    the n bounds."""
    return evaluations * (4 * R + 4 * R + R / 8) + extractions * 8 * n


def celf_refresh_bytes(n, R, refreshes, refreshed):
    """Bytes of the bound refreshes, a choice of this design rather than work
    the method requires: each scans the n bounds and chosen flags, and the
    vertices whose bound reaches the best known exact gain are re-evaluated."""
    return refreshed * (4 * R + 4 * R + R / 8) + refreshes * 9 * n


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


def measure(name, w, xadj, adj, steps, warmup, world, detail):
    """Device-timed steps of one workload (inputs resident). Returns the
    record and, when detail is set, the per-kernel breakdown."""
    import torch

    import paper_2008_03095_gb300 as im

    rank, _, local_rank = dist_env()
    dev = torch.device("cuda", local_rank)
    n = xadj.shape[0] - 1
    m = adj.shape[0] // 2
    R, K, ps, seed = w["R"], w["K"], list(w["ps"]), w["rng_seed"]
    stream = torch.cuda.current_stream()
    im.im_set_stream(stream)

    g = im.im_graph_create(xadj, adj)
    d_seeds = torch.empty((len(ps), K), dtype=torch.int32, device=dev)
    d_sigma = torch.empty((len(ps), K), dtype=torch.int64, device=dev)
    d_spread = torch.empty((len(ps),), dtype=torch.int64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # The queries of a step are independent: each runs on its own stream with
    # its own workspace, forked from and joined back to the launching stream.
    q_streams = [torch.cuda.Stream(device=dev) for _ in ps]
    q_ws = [im.im_workspace_create(g, R) for _ in ps]
    ws = q_ws[0]

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

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    for w_ in q_ws:
        im.im_workspace_status(w_)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank) if detail else None
    if clocks:
        clocks.start()
    launches0 = im.im_kernel_launches()
    total_ms = timed_steps(steps)
    launches = im.im_kernel_launches() - launches0
    clock_info = clocks.stop() if clocks else None
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
    nprof = max(1, min(steps, 10))
    im.im_workspace_stats(ws)
    im.im_profile_enable(True)
    serial_ms = timed_steps(nprof, step_serial)
    prof = im.im_profile_read()
    by_p = {}
    for i, p in enumerate(ps):
        im.im_profile_read()
        im.im_workspace_stats(ws)
        for _ in range(nprof):
            flush.zero_()
            im.im_select_seeds_async(g, ws, K, R, p, seed, d_seeds[i], d_sigma[i])
            im.im_estimate_spread_async(g, ws, d_seeds[i], K, R, p, seed, d_spread[i:i + 1])
        pp = im.im_profile_read()
        st = im.im_workspace_stats(ws)
        by_p[str(p)] = {"avg_us": {k: round(v[0] / v[1] * 1e3, 2) for k, v in pp.items() if v[1]},
                        "per_query": {k: v / nprof for k, v in st.items()}}
    im.im_profile_enable(False)
    im.im_set_stream(None)
    for w_ in q_ws:
        w_.close()
    g.close()
    del flush
    torch.cuda.empty_cache()

    peak, peak_kind = measured_peaks()
    units_per_step = len(ps) * 2 * m * R
    rec = {"ms_per_step": total_ms / steps, "steps": steps, "warmup": warmup,
           "value": job_throughput(units_per_step * steps, total_ms / 1e3, world),
           "ms_per_step_one_stream": serial_ms / nprof, "gpu_launches": int(launches),
           "consistent_spread": consistent}
    expected = stored_oracle(name)
    if expected:
        rec["parity_vs_stored_oracle"] = bool(all(
            p in expected and np.array_equal(seeds_h[i], expected[p][0])
            and np.array_equal(sigma_h[i], expected[p][1]) for i, p in enumerate(ps)))

    # The component pipeline (label init, fused sample + union, size memo,
    # first gains) against its algorithmic floor 8m + 4(n+1) + 20nR bytes per
    # query: the CSR once, labels written, read for sizes, sizes written,
    # labels and sizes read for the first gains.
    cc_phases = ("prep", "union", "compress", "gains")
    cc_us = sum(prof[ph][0] for ph in cc_phases) * 1e3 / (nprof * len(ps))
    cc_bytes = 8 * m + 4 * (n + 1) + 20 * n * R
    cc_gbs = cc_bytes / (cc_us / 1e6) / 1e9
    rec["component_pipeline"] = {
        "phases": list(cc_phases), "us_per_query": cc_us, "bytes_per_query": cc_bytes,
        "achieved_gbs": cc_gbs, "frac": cc_gbs / peak, "peak": peak, "peak_kind": peak_kind,
        "frac_of": "measured" if peak_kind == "measured" else "fallback"}
    per_kernel = {k: {"total_ms": v[0], "launches": v[1],
                      "avg_us": (v[0] / v[1] * 1e3) if v[1] else None} for k, v in prof.items()}
    tot = sum(v[0] for v in prof.values())
    for k in per_kernel:
        per_kernel[k]["share"] = prof[k][0] / tot if tot else None
    rec["per_kernel"] = per_kernel
    rec["per_p"] = by_p
    if not detail:
        return rec, (seeds_h, sigma_h, spread_h)

    rec["clocks"] = clock_info
    # Roofline of the dominant kernel (largest share of device time). The
    # spread's hand-over runs the select path's union again (phase
    # spread_union): it counts toward that kernel when every query handed
    # over, so that every launch did the full work.
    handed_over = all(by_p[str(p)]["per_query"].get("spread_components", 0) >= 1 for p in ps)
    kern = {}
    for ph, (ms, cnt) in prof.items():
        k = {"spread_union": "union"}.get(ph, ph)
        if k != ph and not handed_over:
            continue
        a, c = kern.get(k, (0.0, 0))
        kern[k] = (a + ms, c + cnt)
    dominant = max(kern, key=lambda k: kern[k][0])
    T = {p: im.im_sampling_threshold(p) for p in ps}
    avg_s = kern[dominant][0] / kern[dominant][1] / 1e3
    roof = {"kernel": KERNEL_OF_PHASE.get(dominant, "k_" + dominant), "bound": "hbm",
            "peak": peak, "unit": "GB/s",
            "peak_kind": peak_kind, "avg_launch_us": avg_s * 1e6, "launches": kern[dominant][1],
            "share_of_device_time": kern[dominant][0] / tot if tot else None}
    if dominant == "celf":
        q = [by_p[str(p)]["per_query"] for p in ps]
        mb = statistics.mean(celf_method_bytes(n, R, x["celf_evaluations"], x["celf_extractions"])
                             for x in q)
        rb = statistics.mean(celf_refresh_bytes(n, R, x["celf_refreshes"], x["celf_refreshed"])
                             for x in q)
        roof.update(bytes_per_launch=mb, refresh_bytes_per_launch=rb,
                    achieved=mb / avg_s / 1e9,
                    note="method bytes only (exact gain evaluations E*(8R + R/8) plus prefix "
                         "extractions X*8n); the dense refreshes' bytes are given apart; "
                         "latency-bound: the driver's cluster runs the sequential rounds; "
                         "no DRAM counters: the profiler is not run on this cooperative "
                         "cluster launch",
                    traffic=None)
    else:
        if dominant == "union":
            b = statistics.mean(algorithmic_bytes("union", n, g_m_up(xadj, adj), R, T[p])
                                for p in ps)
        else:
            b = algorithmic_bytes(dominant, n, 0, R, 0)
        if b is None:  # spread: per-level work varies; report its time only
            roof.update(bound="latency", achieved=None, bytes_per_launch=None, traffic=None)
        else:
            roof.update(bytes_per_launch=b, achieved=b / avg_s / 1e9,
                        traffic=committed_traffic(roof["kernel"], name))
    if roof.get("achieved") is not None:
        roof["frac"] = roof["achieved"] / peak
        roof["frac_of"] = "measured" if peak_kind == "measured" else "fallback"
    else:
        roof["frac"] = None
    rec["roofline"] = roof
    hbm = {}
    for ph in ("prep", "compress", "gains", "spread_cc"):
        if prof[ph][1] and (ph != "spread_cc" or handed_over):
            b = algorithmic_bytes(ph, n, 0, R, 0)
            a = b / (prof[ph][0] / prof[ph][1] / 1e3) / 1e9
            kn = KERNEL_OF_PHASE.get(ph, "k_" + ph)
            hbm[kn] = {"achieved_gbs": a, "frac": a / peak, "bytes_per_launch": b,
                       "traffic": committed_traffic(kn, name)}
    rec["hbm_kernels"] = hbm
    return rec, (seeds_h, sigma_h, spread_h)


def run_e2e(args, xadj, adj, w, world):
    """Same metric through the blocking C ABI with host buffers: graph upload
    from pinned host memory, select (host outputs), spread (host seeds), free."""
    import torch

    import paper_2008_03095_gb300 as im

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
    units = len(ps) * 2 * m * R * args.e2e_steps
    h2d = 4 * (n + 1) + 8 * m + len(ps) * K * 4
    d2h = len(ps) * (K * 4 + K * 8 + 8)
    return {"value": job_throughput(units, dt, world), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
            "ms_per_step": dt * 1e3 / args.e2e_steps,
            "path": "im_graph_create (pinned host CSR) + im_select_seeds + im_estimate_spread "
                    "per p + im_graph_destroy"}


def run_cpu_baseline(name, xadj, adj, w):
    """The oracle as it stands on the host cores: single-threaded and its
    OpenMP build on all cores, each on one step of the workload restricted to
    the first few simulations (CPU_LANES), scaled per sampled edge visit."""
    import oracle

    m = adj.shape[0] // 2
    l1, lall = CPU_LANES.get(name, (8, 64))
    out = {}
    spread = name not in ORACLE_SELECT_ONLY
    for label, lanes, omp in (("single_thread", l1, False), ("all_cores", lall, True)):
        oracle.use_all_cores(omp)
        t0 = time.perf_counter()
        oracle_step(oracle, xadj, adj, w, lanes, spread)
        dt = time.perf_counter() - t0
        out[label] = {"value": len(w["ps"]) * 2 * m * lanes / dt / 1e9, "unit": UNIT,
                      "cores": oracle.threads(), "lanes": lanes, "seconds": dt}
    oracle.use_all_cores(False)
    main = out["all_cores"]
    return {"value": main["value"], "unit": UNIT, "cores": main["cores"], "kind": "oracle",
            "sample": "one step (%s, K=%d, p in %s) on the first %d of R=%d "
                      "simulations, OpenMP build on all host cores; single thread on the "
                      "first %d: %.4g %s" % (oracle_step_kind(name), w["K"], list(w["ps"]),
                                             lall, w["R"], l1, out["single_thread"]["value"],
                                             UNIT),
            "single_thread": out["single_thread"], "all_cores": out["all_cores"],
            "nproc": os.cpu_count(), "cpu": cpu_model()}


def _instance_graph(inst):
    from paper_2008_03095_gb300 import synth
    return synth.instance_graph(inst)


def batch_graphs(count):
    """The uneven instances of the batched recipe and their graphs, built in
    a spawn pool of host processes (started before any CUDA call)."""
    import multiprocessing as mp

    from paper_2008_03095_gb300 import synth
    inst = synth.batched_instances(count=count)
    procs = max(1, min(16, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        graphs = pool.map(_instance_graph, inst, chunksize=4)
    return inst, graphs


def serve_graphs():
    """The serving pool's graphs: 64 of the batched recipe (parameters from
    PCG64(50)) and the 2,000-, 15,233- and 37,154-vertex workload graphs."""
    import multiprocessing as mp

    from paper_2008_03095_gb300 import synth
    inst = synth.batched_instances(count=64, seed=50)
    procs = max(1, min(16, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        graphs = pool.map(_instance_graph, inst, chunksize=2)
    for name in ("powerlaw_n2000", "powerlaw_n15233", "powerlaw_n37154"):
        graphs.append(synth.workload_graph(name))
    return graphs


def run_batch(args, inst, graphs, world):
    """The batched persistent launch of all instances against the same
    queries one at a time (im_select_seeds_async on one stream, a workspace
    per graph made beforehand): device time with CUDA events, W warm-up runs,
    K timed runs each; the autotuner picks the tiling first."""
    import torch

    import paper_2008_03095_gb300 as im

    dev = torch.device("cuda", dist_env()[2])
    handles = [im.im_graph_create(x, a) for x, a in graphs]
    queries = [dict(graph=i, K=x["K"], R=x["R"], p=x["p"], rng_seed=x["rng_seed"])
               for i, x in enumerate(inst)]
    units = sum(2 * x["m"] * x["R"] for x in inst)
    stream = torch.cuda.current_stream()
    im.im_set_stream(stream)
    b = im.im_batch_create(handles, queries)
    t0 = time.perf_counter()
    im.im_batch_autotune(b, 2)
    tune_s = time.perf_counter() - t0
    wss = [im.im_workspace_create(h, q["R"]) for h, q in zip(handles, queries)]
    d_seeds = [torch.empty(q["K"], dtype=torch.int32, device=dev) for q in queries]
    d_sigma = [torch.empty(q["K"], dtype=torch.int64, device=dev) for q in queries]

    def solo():
        for i, q in enumerate(queries):
            im.im_select_seeds_async(handles[i], wss[i], q["K"], q["R"], q["p"], q["rng_seed"],
                                     d_seeds[i], d_sigma[i])

    def timed(fn):
        for _ in range(max(1, args.warmup // 2)):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.batch_steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts

    launches0 = im.im_kernel_launches()
    t_batch = timed(lambda: im.im_batch_run_async(b))
    batch_launches = (im.im_kernel_launches() - launches0) // (args.batch_steps + max(1, args.warmup // 2))
    seeds, sigma, status = im.im_batch_results(b, check=False)
    # the lazy-greedy items (one SM each): whole item and bound refreshes, in
    # SM cycles (converted at the 2070 MHz the bench runs at)
    item_cyc, ref_cyc = [], []
    for i in range(len(queries)):
        st = im.im_batch_query_stats(b, i)
        item_cyc.append(st["celf_cycles_eval"])
        ref_cyc.append(st["celf_cycles_refresh"])
    slowest = int(np.argmax(item_cyc))
    cyc = im.im_batch_phase_cycles(b)  # of the last timed run
    t_solo = timed(solo)
    same = bool(np.all(status == 0)) and all(
        np.array_equal(seeds[i], d_seeds[i].cpu().numpy())
        and np.array_equal(sigma[i], d_sigma[i].cpu().numpy().astype(np.uint64))
        for i in range(len(queries)))
    info = im.im_batch_info(b)
    im.im_set_stream(None)
    for w_ in wss:
        w_.close()
    b.close()
    for h in handles:
        h.close()
    torch.cuda.empty_cache()
    mb, ms_ = statistics.median(t_batch), statistics.median(t_solo)
    return {"queries": len(queries), "units": units, "n_total": int(sum(x["n"] for x in inst)),
            "m_total": int(sum(x["m"] for x in inst)), "label_bytes": info["device_bytes"],
            "work_items": info["items"], "launches_per_run": int(batch_launches),
            "autotune_s": tune_s, "batch_ms": mb, "one_at_a_time_ms": ms_,
            "value": units / (mb / 1e3) / 1e9, "value_one_at_a_time": units / (ms_ / 1e3) / 1e9,
            "speedup": ms_ / mb, "unit": UNIT, "results_equal_one_at_a_time": same,
            "schedule_group": info["schedule"],
            "slowest_celf_item_ms": item_cyc[slowest] / 2.07e6,
            "slowest_celf_item_refresh_ms": ref_cyc[slowest] / 2.07e6,
            "slowest_celf_item_query": {k: inst[slowest][k] for k in ("n", "m", "R", "K", "p")},
            "celf_items_ms_sum": sum(item_cyc) / 2.07e6,
            "sm_ms_per_phase": {"work": {k: v / 2.07e6 for k, v in cyc["work"].items()},
                                "wait": {k: v / 2.07e6 for k, v in cyc["wait"].items()},
                                "help": cyc["help"] / 2.07e6},
            "recipe": "256 Chung-Lu graphs: n log-uniform [500, 200000], m/n U[2, 15], exponent "
                      "U[2, 3], p log-uniform [0.001, 0.1], R in {256, 1024, 2048}, K U{5..100}, "
                      "parameters from PCG64(40), graph i seed 1000 + i"}


def serve_queries(rng, pool_n, count):
    """The serving recipe's query stream: 70 % select / 30 % spread of a random
    K-subset, K ~ U{5..100} (at most n), R in {256, 1024, 2048}, p
    log-uniform in [0.001, 0.1], over the pool's graphs uniformly."""
    out = []
    for _ in range(count):
        gi = int(rng.integers(0, len(pool_n)))
        n = pool_n[gi]
        K = int(min(rng.integers(5, 101), n))
        R = int(rng.choice([256, 1024, 2048]))
        p = float(np.exp(rng.uniform(np.log(0.001), np.log(0.1))))
        seed = int(rng.integers(0, 1 << 31))
        if rng.random() < 0.7:
            out.append(dict(kind=0, graph=gi, K=K, R=R, p=p, rng_seed=seed))
        else:
            out.append(dict(kind=1, graph=gi, K=K, R=R, p=p, rng_seed=seed,
                            seeds=rng.choice(n, size=K, replace=False).astype(np.int32)))
    return out


def pct(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def run_serve(args, pool_graphs):
    """Serving with continuous batching against serial execution. The pool:
    64 graphs of the batched recipe plus the 2,000-, 15,233- and
    37,154-vertex workload graphs, resident. For each offered load, `--serve`
    queries arrive as a Poisson stream in real time; latency = completion -
    arrival. Serial: the same queries' service times measured one at a time
    (blocking calls, back to back), then queued FIFO under the same arrivals
    (start = max(arrival, previous finish))."""
    import paper_2008_03095_gb300 as im

    handles = [im.im_graph_create(x, a) for x, a in pool_graphs]
    pool_n = [x.shape[0] - 1 for x, _ in pool_graphs]
    rng = np.random.default_rng(50)
    qs = serve_queries(rng, pool_n, args.serve)
    sv = im.im_server_create(handles, slots=16, memory_budget=160 << 30)

    def submit(q):
        return im.im_server_submit(sv, q["kind"], q["graph"], q["K"], q["R"], q["p"],
                                   q["rng_seed"], 0, q.get("seeds"))

    # warm-up: one workspace per graph at the largest R
    for gi in range(len(handles)):
        im.im_server_wait(sv, submit(dict(kind=0, graph=gi, K=5, R=2048, p=0.01, rng_seed=1)))
    # serial service times
    service = []
    for q in qs:
        t0 = time.perf_counter()
        if q["kind"] == 0:
            im.im_select_seeds(handles[q["graph"]], q["K"], q["R"], q["p"], q["rng_seed"])
        else:
            im.im_estimate_spread(handles[q["graph"]], q["seeds"], q["R"], q["p"], q["rng_seed"])
        service.append(time.perf_counter() - t0)
    out = {"queries_per_load": len(qs), "pool_graphs": len(handles), "slots": 16,
           "serial_mean_service_ms": 1e3 * float(np.mean(service)), "loads": {}}
    for rate in [float(r) for r in args.serve_rates.split(",")]:
        gaps = np.random.default_rng(int(rate)).exponential(1.0 / rate, size=len(qs))
        arrive = np.cumsum(gaps)
        tickets = []
        t_start = time.perf_counter()
        for q, a in zip(qs, arrive):
            while time.perf_counter() - t_start < a:
                time.sleep(min(0.0005, max(0.0, a - (time.perf_counter() - t_start))))
            tickets.append((submit(q), time.perf_counter()))
        lat, done_t, failed = [], [], []
        for i, (t, t_sub) in enumerate(tickets):
            try:
                _, _, times = im.im_server_wait(sv, t)
            except im.IMError as err:  # recorded and re-run alone below
                failed.append({"index": i, "code": err.code, "message": str(err),
                               "query": {k: v for k, v in qs[i].items() if k != "seeds"}})
                continue
            lat.append(times[2] - times[0])
            done_t.append(times[2])
        for f in failed:  # alone, through the server and through the blocking call
            q = qs[f["index"]]
            try:
                im.im_server_wait(sv, submit(q))
                f["alone_server"] = "ok"
            except im.IMError as err:
                f["alone_server"] = err.code
            try:
                if q["kind"] == 0:
                    im.im_select_seeds(handles[q["graph"]], q["K"], q["R"], q["p"], q["rng_seed"])
                else:
                    im.im_estimate_spread(handles[q["graph"]], q["seeds"], q["R"], q["p"],
                                          q["rng_seed"])
                f["alone_blocking"] = "ok"
            except im.IMError as err:
                f["alone_blocking"] = err.code
        span = max(done_t) - min(dt - l for dt, l in zip(done_t, lat))
        fin, ser_lat = 0.0, []
        for a, sv_t in zip(arrive, service):
            fin = max(a, fin) + sv_t
            ser_lat.append(fin - a)
        out["loads"][str(int(rate))] = {
            "offered_qps": rate, "p50_ms": 1e3 * pct(lat, 50), "p99_ms": 1e3 * pct(lat, 99),
            "throughput_qps": len(lat) / span,
            "serial_p50_ms": 1e3 * pct(ser_lat, 50), "serial_p99_ms": 1e3 * pct(ser_lat, 99),
            "serial_throughput_qps": len(qs) / max(fin, float(arrive[-1])),
            "failed": failed}
    st = im.im_server_stats(sv)
    out["server_stats"] = {k: st[k] for k in ("in_flight_peak", "queue_peak", "ws_created",
                                               "ws_evicted", "pool_bytes_peak")}
    sv.close()
    for h in handles:
        h.close()
    return out


def run_ours(args, world):
    import torch

    import paper_2008_03095_gb300 as im
    from paper_2008_03095_gb300 import build as lib_build
    from paper_2008_03095_gb300 import synth

    rank, _, local_rank = dist_env()
    lib_build.build()
    im.lib()
    torch.cuda.set_device(local_rank)
    w = synth.WORKLOADS[args.workload]
    xadj, adj = synth.workload_graph(args.workload)
    rec, results = measure(args.workload, w, xadj, adj, args.steps, args.warmup, world, True)
    out = {
        "metric": METRIC, "value": rec.pop("value"), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec.pop("ms_per_step"),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded Chung-Lu / clustered graphs shaped like the paper's "
                "networks; no dataset)",
        "config": workload_config(args.workload, xadj, adj, w),
        "gpu_launches": rec.pop("gpu_launches"),
    }
    out.update(rec)
    out["select_plus_spread_ms_per_query"] = out["ms_per_step"] / len(w["ps"])
    out["e2e"] = run_e2e(args, xadj, adj, w, world)
    if not args.no_extra:
        extra = {}
        for name in EXTRA_WORKLOADS:
            if name == args.workload:
                continue
            we = synth.WORKLOADS[name]
            xe, ae = synth.workload_graph(name)
            r, _ = measure(name, we, xe, ae, args.extra_steps, 2, world, False)
            r["config"] = workload_config(name, xe, ae, we)
            r["unit"] = UNIT
            extra[name] = r
        out["extra_workloads"] = extra
    out["paper_context"] = ("no paper number for this graph; the paper's largest comparable "
                            "runs (Table 4, 2x Xeon E5-2620v4, 16 threads, K=50, p=0.01): "
                            "Amazon 262k v 2.09 s, NetHEP 15k v 0.08 s, NetPhy 37k v 0.36 s; "
                            "R not stated")
    return out, (xadj, adj, w, results)


def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    from paper_2008_03095_gb300 import synth

    if args.impl == "reference":
        if rank != 0:
            return 0
        w = synth.WORKLOADS[args.workload]
        xadj, adj = synth.workload_graph(args.workload)
        print(json.dumps(run_reference(args, xadj, adj, w)))
        return 0

    import torch

    if world > 1:
        import datetime
        torch.distributed.init_process_group(
            backend="nccl" if torch.cuda.is_available() else "gloo",
            timeout=datetime.timedelta(minutes=10))
    batch_inst = batch_graphs(args.batch) if args.batch > 0 else None
    serve_pool = serve_graphs() if args.serve > 0 else None
    out, (xadj, adj, w, results) = run_ours(args, world)
    if batch_inst is not None:
        out["batched"] = run_batch(args, batch_inst[0], batch_inst[1], world)
    if serve_pool is not None:
        out["serving"] = run_serve(args, serve_pool)
    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = run_cpu_baseline(args.workload, xadj, adj, w)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
