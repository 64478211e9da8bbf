#!/usr/bin/env python3
"""Benchmark: candidate windows/s of EAPrunedDTW subsequence search on GB300.

One step = the large workload: a Gaussian random walk of 20,000,000 FP32 points
(seed 0) searched by four random-walk queries of length 1024 (seeds 1-4), each
once with w = 103 (10%, LB_Kim -> LB_Keogh EQ -> EC -> EAPrunedDTW) and once
with w = 1024 (unconstrained, no lower bounds): 8 searches, k = 1.

Prints one JSON line (rank 0).  `value` is whole-job candidate windows/s with
the inputs resident in HBM; `e2e` is the same metric with the reference and
queries copied from pinned host memory and the results read back every step.
`--impl reference` times the CPU oracle on a bounded sample of the same
workload instead.

Two more objects on the same line (rank 0, one GPU): `batched` times the
batched search (eapdtw_search_batch: one graph-captured launch sequence) and
the one-query-per-call path on the same sample of the batched mix (queries of
uneven lengths and windows, each against 8 references); `serving` runs the
serving loop (continuous batching) against a resident 1e8-point reference,
first with every request submitted at once, then with Poisson arrivals at half
that throughput, and reports p50/p99 latency and queries/s.  `extensions`
measures the absolute-cost search, upper-bound tightening on and off, the
pairwise DTW matrix and 1-NN classification.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_DEFAULT = 20_000_000
M = 1024
QUERY_SEEDS = (1, 2, 3, 4)
SEARCHES = [(103, False), (1024, True)]  # (w, no lower bounds)
METRIC = "candidate windows/s"
GOLDEN = os.path.join(ROOT, "tests", "golden", "bench_large_oracle.json")
# Rows per thread of the DP-cell throughput probe (eapdtw_cell_peak), whose
# fastest mode is the roofline's peak.
PEAK_STEPS = 1 << 18
PEAK_MODES = (0, 1, 2, 3)
# DRAM bytes (read + write) of the dominant search kernel per search, from an
# ncu capture of the kernel as built (scaled from n = 1e7 to the workload's
# 19,998,977 windows), or None when the kernel has changed since the last
# capture.  The last one (207.8 MB for 9,998,977 windows, 20.8 B per window)
# predates keeping the row fill's inputs in shared memory.
TRAFFIC_BYTES_PER_SEARCH = None
# CPU baseline sample (oracle): windows of the cascade (w=103) and nolb (w=1024) searches
CPU_SAMPLE = {"cascade_windows": 2_000_000, "nolb_windows": 200_000, "query_seed": 1}


def workload_desc(n):
    return (f"large: random walk n={n} (FP32, seed 0); 4 random-walk queries m={M} (seeds 1-4); "
            f"each searched with w=103 + LB_Kim/LB_Keogh cascade and with w=1024 (unconstrained, "
            f"no lower bounds); k=1")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of every rank's x: the slowest replica sets the job's time.
    With one rank, x itself (no process group needed)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_total: float, ms: float) -> float:
    """Whole-job throughput: the units of the whole job (each window of each
    search is searched by exactly one rank) over the slowest rank's time per
    step."""
    return units_total / (ms / 1e3)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_golden(n):
    try:
        with open(GOLDEN) as f:
            g = json.load(f)
    except (OSError, ValueError):
        return None
    if f"n={n}" not in g.get("workload", ""):
        return None
    want = {(s, w, not nolb) for s in QUERY_SEEDS for (w, nolb) in SEARCHES}
    have = {(e["query_seed"], e["w"], e["lower_bounds"]): e for e in g.get("searches", [])}
    if not want.issubset(have):
        return None
    return have


def cpu_baseline(n_threads=None):
    """The oracle (FP64 C cascade) on a bounded sample of the workload."""
    import oracle as O
    from paper_2010_05371_gb300 import synth
    nt = n_threads or os.cpu_count() or 1
    Q = synth.random_walk(M, CPU_SAMPLE["query_seed"])
    nc, nn = CPU_SAMPLE["cascade_windows"], CPU_SAMPLE["nolb_windows"]
    R = synth.random_walk(max(nc, nn) + M - 1, 0)
    t0 = time.perf_counter()
    O.search_cascade(Q, R[:nc + M - 1], 103, 1, use_lb=True, nthreads=nt)
    t1 = time.perf_counter()
    O.search_cascade(Q, R[:nn + M - 1], 1024, 1, use_lb=False, nthreads=nt)
    t2 = time.perf_counter()
    rate_c, rate_n = nc / (t1 - t0), nn / (t2 - t1)
    # the step has as many cascade windows as nolb windows
    rate = 2.0 / (1.0 / rate_c + 1.0 / rate_n)
    return {"value": rate, "unit": "windows/s", "cores": nt, "kind": "oracle",
            "sample": (f"oracle FP64 C search, query seed 1: w=103 cascade over the first {nc} windows "
                       f"({rate_c:.3g} windows/s) and w=1024 nolb over the first {nn} windows "
                       f"({rate_n:.3g} windows/s), combined for the step's equal mix"),
            "seconds": round(t2 - t0, 2)}


# Batched sample: the 1,024-query x 8-reference mix, cut to --batch-queries
# queries (every query against every reference).
BATCH_REF_SEED, BATCH_QUERY_SEED = 3, 2
BATCH_FULL_QUERIES = 1024   # queries of the full mix (each against the 8 references)
BATCH_REPEATS = 3
# Serving: a resident random walk of 1e8 points; requests with m log-uniform in
# [64, 4096], window ratio uniform in [0, 0.5], k in {1, 5}.
SERVE_N, SERVE_ARRIVAL_SEED, SERVE_QUERY_SEED = 100_000_000, 4, 5
SERVE_RATES = (0.25, 0.5, 0.9)   # Poisson arrival rates, as fractions of the saturated throughput


def batched_mix(nq, seed=BATCH_QUERY_SEED):
    """Parameters of the batched mix's nq queries in draw order: (m, w, ecg, k)
    with m log-uniform in [64, 2048], window ratio uniform in [0, 1], random walk
    or ECG-like by a coin flip, k in {1, 5}."""
    import math
    rq = np.random.default_rng(seed)
    out = []
    for _ in range(nq):
        m = int(round(math.exp(rq.uniform(math.log(64), math.log(2048)))))
        ratio = rq.uniform(0.0, 1.0)
        w = int(math.ceil(ratio * m))
        ecg = rq.random() < 0.5
        k = 1 if rq.random() < 0.5 else 5
        out.append((m, w, ecg, k, ratio))
    return out


def _stratum(m, ratio):
    """Stratum of a query of the mix: 4 log-uniform length buckets x 4 window-ratio buckets."""
    import math
    lb = min(3, int((math.log(m) - math.log(64)) / ((math.log(2048) - math.log(64)) / 4)))
    return lb * 4 + min(3, int(ratio * 4))


def sample_strata(mix, nq):
    """The batched sample: the first random-walk and the first ECG-like query
    of each (length x window-ratio stratum), in draw order, at most nq of them;
    and each (stratum, kind)'s count in the whole mix (the weights of the
    full-mix estimate)."""
    counts, first = {}, {}
    for q, (m, w, ecg, k, ratio) in enumerate(mix):
        key = (_stratum(m, ratio), bool(ecg))
        counts[key] = counts.get(key, 0) + 1
        first.setdefault(key, q)
    return sorted(first.values())[:nq], counts


def batched_section(args, dev):
    """Batched search (one graph-captured launch sequence over all items)
    against the one-query-per-call path on the same items: a stratified sample
    of the 1,024-query mix (the first random-walk and the first ECG-like query
    of each of 16 length x window-ratio strata, each against the 8
    references), and the full mix's time estimated from it: each sampled
    query's one-call time and the time of its 8 items as a batch of their own,
    weighted by its (stratum, kind)'s share of the 1,024 queries."""
    import math
    import torch
    from paper_2010_05371_gb300 import api, synth
    rr = np.random.default_rng(BATCH_REF_SEED)
    lens = [int(round(math.exp(rr.uniform(math.log(1e5), math.log(1e7))))) for _ in range(8)]
    refs = [torch.from_numpy(synth.random_walk(n, 100 + j).astype(np.float32)).to(dev)
            for j, n in enumerate(lens)]
    mix = batched_mix(BATCH_FULL_QUERIES)
    picked, counts = sample_strata(mix, args.batch_queries)
    if args.batch_strata:   # profiling aid: only these of the sampled strata
        picked = [picked[int(j)] for j in args.batch_strata.split(",")]
    queries = []
    for q in picked:
        m, w, ecg, k, ratio = mix[q]
        qn = synth.ecg_query(m, 1000 + q) if ecg else synth.random_walk(m, 1000 + q)
        queries.append((q, torch.from_numpy(np.asarray(qn, np.float32)).to(dev), w, k))
    ctx = api.Context(dev.index or 0)
    ids = [ctx.register(R) for R in refs]
    items = [(Q, rid, w, k) for (q, Q, w, k) in queries for rid in ids]
    item_query = [q for (q, Q, w, k) in queries for rid in ids]
    windows = sum(refs[rid].numel() - Q.numel() + 1 for (Q, rid, w, k) in items)
    ctx.search_batch(items, 5)            # warm-up: graph capture, envelope tables
    torch.cuda.synchronize()
    # the built-in rule (no tuning table), then the autotuned table
    _, _, cnt_fixed = ctx.search_batch(items, 5, return_counters=True)
    torch.cuda.synchronize()
    fixed_s = cnt_fixed["ns_total"] / 1e9
    t0 = time.perf_counter()
    tuned = ctx.autotune(items, sample_windows=1 << 20)   # first-level tile and check interval per signature
    tune_s = time.perf_counter() - t0
    tuning = ctx.tuning_table()
    dev_ms, host_s = [], []
    cnt = None
    for _ in range(BATCH_REPEATS):
        t0 = time.perf_counter()
        bi, bd, cnt = ctx.search_batch(items, 5, return_counters=True)
        torch.cuda.synchronize()
        host_s.append(time.perf_counter() - t0)
        dev_ms.append(cnt["ns_total"] / 1e6)
    tb = statistics.median(dev_ms) / 1e3
    big = max(range(len(refs)), key=lambda j: refs[j].numel())
    api.subseq_search(queries[0][1], refs[big], queries[0][2], 1)   # warm-up of the plain scratch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain, plain_ns = [], []
    for (Q, rid, w, k) in items:
        pi, pd, pc = api.subseq_search(Q, refs[rid], w, k, return_counters=True)
        plain.append((pi, pd))
        plain_ns.append(pc["ns_total"])
    torch.cuda.synchronize()
    tp_host = time.perf_counter() - t0
    tp = sum(plain_ns) / 1e9
    mism = sum(0 if torch.equal(pd, bd[i, :k]) else 1
               for i, ((Q, rid, w, k), (pi, pd)) in enumerate(zip(items, plain)))
    # each sampled query's items as a batch of their own (device time; the
    # launch sequence is captured and its kernels loaded by the runs above)
    per_query_ns = {}
    for q, ns in zip(item_query, plain_ns):
        per_query_ns[q] = per_query_ns.get(q, 0) + ns
    per_query_batch_ns = {}
    for q in picked:
        own = [it for it, iq in zip(items, item_query) if iq == q]
        _, _, c1 = ctx.search_batch(own, 5, return_counters=True)
        per_query_batch_ns[q] = c1["ns_total"]
    torch.cuda.synchronize()
    # the full mix: each (stratum, kind)'s share of the 1,024 queries x its sampled query's times
    weight = {q: counts[(_stratum(mix[q][0], mix[q][4]), bool(mix[q][2]))] for q in picked}
    est_plain_s = sum(weight[q] * per_query_ns[q] for q in picked) / 1e9
    est_batch_s = sum(weight[q] * per_query_batch_ns[q] for q in picked) / 1e9
    wins = sum(1 for q in picked if per_query_batch_ns[q] < per_query_ns[q])
    full_windows = sum(sum(n - m + 1 for n in lens) for (m, w, ecg, k, ratio) in mix)
    ctx.close()
    return {
        "config": (f"batched mix: {len(picked)} queries, the first random-walk and the first ECG-like query of each "
                   f"length x window-ratio stratum of the "
                   f"{BATCH_FULL_QUERIES}-query mix (m log-uniform 64-2048, window ratio uniform 0-1, random walk "
                   f"or ECG-like, k in {{1,5}}, seed {BATCH_QUERY_SEED}) x 8 random-walk references (n log-uniform "
                   f"1e5-1e7, seed {BATCH_REF_SEED}), every query against every reference"),
        "items": len(items), "windows": windows,
        "timing": (f"device time (CUDA events) of the batched launch sequence, median of {BATCH_REPEATS} "
                   f"after 1 warm-up; the one-call path's device time summed over its calls"),
        "autotune": (f"{tuned} signatures tuned in {tune_s:.1f} s (not timed): "
                     f"{sum(1 for v in tuning.values() if v[1])} at the doubled check interval"),
        "fixed_rule_s": round(fixed_s, 4), "tuned_over_fixed": fixed_s / tb,
        "batched_s": round(tb, 4), "batched_s_repeats": [round(x / 1e3, 4) for x in dev_ms],
        "batched_host_s": round(statistics.median(host_s), 4),
        "plain_s": round(tp, 4), "plain_host_s": round(tp_host, 4),
        "batched_windows_per_s": windows / tb, "plain_windows_per_s": windows / tp,
        "batched_queries_per_s": len(items) / tb, "plain_queries_per_s": len(items) / tp,
        "speedup": tp / tb, "executed_cells_per_s": cnt["cells"] / tb,
        "identical_to_plain": f"{len(items) - mism}/{len(items)} items bit-identical distances",
        "per_query": {"queries": len(picked), "batch_faster": wins,
                      "speedup_median": statistics.median(per_query_ns[q] / per_query_batch_ns[q] for q in picked)},
        "full_mix_estimate": {
            "queries": BATCH_FULL_QUERIES, "items": BATCH_FULL_QUERIES * len(refs), "windows": full_windows,
            "plain_s": round(est_plain_s, 2), "batched_s": round(est_batch_s, 2),
            "speedup": est_plain_s / est_batch_s,
            "basis": ("(stratum, kind) counts of the full mix x that (stratum, kind)'s sampled query: its one-call "
                      "times, and its items as a batch of their own (device time)")},
    }


def serving_section(args, dev):
    """Serving loop against a resident 1e8-point reference: every request at
    once (saturated), the same requests through the one-query-per-call path
    (plain), and Poisson arrivals at swept fractions of the saturated rate."""
    import math
    import torch
    from paper_2010_05371_gb300 import api, synth
    n = args.serve_n
    R = torch.from_numpy(synth.random_walk(n, 0).astype(np.float32)).to(dev)
    ctx = api.Context(dev.index or 0)
    rid = ctx.register(R)
    rq = np.random.default_rng(SERVE_QUERY_SEED)

    def draw(count, base):
        out = []
        for i in range(count):
            m = int(round(math.exp(rq.uniform(math.log(64), math.log(4096)))))
            w = int(math.ceil(rq.uniform(0.0, 0.5) * m))
            k = 1 if rq.random() < 0.5 else 5
            out.append((synth.random_walk(m, base + i).astype(np.float32), w, k))
        return out

    ctx.serve_start(max_active=args.serve_active, chunk_windows=1 << 22)
    warm = draw(2, 90_000)
    for Q, w, k in warm:   # warm-up: graph capture and envelope levels
        h = ctx.submit(Q, rid, w, k)
        while ctx.poll(h, k, timeout_ms=1000) is None:
            pass

    def run(reqs, gaps):
        handles = []
        t0 = time.perf_counter()
        for (Q, w, k), g in zip(reqs, gaps):
            if g > 0:
                time.sleep(g)
            handles.append(ctx.submit(Q, rid, w, k))
        lat, res = [], []
        for h, (Q, w, k) in zip(handles, reqs):
            r = None
            while r is None:
                r = ctx.poll(h, k, timeout_ms=1000)
            lat.append(r[2] / 1e6)
            res.append((r[0], r[1]))
        wall = time.perf_counter() - t0
        return {"requests": len(reqs), "wall_s": round(wall, 3), "queries_per_s": len(reqs) / wall,
                "windows_per_s": sum(n - len(Q) + 1 for Q, w, k in reqs) / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(np.mean(lat))}, res

    reqs = draw(args.serve_requests, 10_000)
    sat, sat_res = run(reqs, [0.0] * len(reqs))
    # the plain path on the same requests: one blocking subseq_search call per
    # request, in submission order (its latency is queueing plus service)
    api.subseq_search(torch.from_numpy(reqs[0][0]).to(dev), R, reqs[0][1], reqs[0][2])   # scratch warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_res, plain_done = [], []
    for Q, w, k in reqs:
        pi, pd = api.subseq_search(torch.from_numpy(Q).to(dev), R, w, k)
        plain_res.append((pi.cpu().numpy(), pd.cpu().numpy()))
        plain_done.append((time.perf_counter() - t0) * 1e3)
    plain_wall = time.perf_counter() - t0
    plain = {"requests": len(reqs), "wall_s": round(plain_wall, 3), "queries_per_s": len(reqs) / plain_wall,
             "p50_ms": float(np.percentile(plain_done, 50)), "p99_ms": float(np.percentile(plain_done, 99))}
    same = sum(int(np.array_equal(sd, pd)) for (si, sd), (pi, pd) in zip(sat_res, plain_res))
    sweep = []
    ra = np.random.default_rng(SERVE_ARRIVAL_SEED)
    for j, frac in enumerate(SERVE_RATES):
        lam = frac * sat["queries_per_s"]
        gaps = list(ra.exponential(1.0 / lam, size=args.serve_poisson_requests))
        gaps[0] = 0.0
        rr = draw(args.serve_poisson_requests, 20_000 + 1000 * j)
        out, _ = run(rr, gaps)
        out["rate_per_s"] = lam
        out["rate_fraction_of_saturated"] = frac
        sweep.append(out)
    st = ctx.serve_stats()
    ctx.serve_stop()
    ctx.close()
    return {
        "config": (f"serving: resident random walk n={n} (FP32, FP64 chunk sums); requests m log-uniform "
                   f"64-4096, window ratio uniform 0-0.5, k in {{1,5}} (query seed {SERVE_QUERY_SEED}); "
                   f"{args.serve_active} state slots, 2^22-window base quantum, cost-ordered rounds"),
        "saturated": sat, "plain_one_call_per_request": plain,
        "served_over_plain_queries_per_s": sat["queries_per_s"] / plain["queries_per_s"],
        "poisson_sweep": sweep, "rounds": st["rounds"],
        "identical_to_plain": f"{same}/{len(reqs)} requests bit-identical distances",
    }


def extensions_section(args, dev, R, Qs):
    """The method's extensions, each measured once after a warm-up (CUDA events
    inside the library for the searches, host clock around the blocking calls
    for the whole-series forms)."""
    import torch
    from paper_2010_05371_gb300 import api, synth
    out = {}
    q = Qs[0]
    nw = R.numel() - q.numel() + 1
    # another elastic cost with DTW's recurrence: |a - b|, no lower bounds
    api.subseq_search(q, R, 1024, 1, no_lb=True, cost=api.COST_ABSOLUTE)
    _, _, c = api.subseq_search(q, R, 1024, 1, no_lb=True, cost=api.COST_ABSOLUTE, return_counters=True)
    out["absolute_cost_search"] = {"config": f"query seed {QUERY_SEEDS[0]}, m={q.numel()}, w=1024, no lower bounds, "
                                             f"cost |a-b|, n={R.numel()}",
                                   "ms": c["ns_total"] / 1e6, "windows_per_s": nw / (c["ns_total"] / 1e9)}
    # upper-bound tightening with the LB_Keogh EQ terms, on and off
    ms = {}
    for tight in (False, True):
        api.subseq_search(q, R, 103, 1, tighten=tight)
        _, _, c = api.subseq_search(q, R, 103, 1, tighten=tight, return_counters=True)
        ms[tight] = (c["ns_total"] / 1e6, c["steps"])
    out["tightening"] = {"config": f"query seed {QUERY_SEEDS[0]}, m={q.numel()}, w=103, cascade, n={R.numel()}",
                         "ms_off": ms[False][0], "ms_on": ms[True][0], "dtw_steps_off": ms[False][1],
                         "dtw_steps_on": ms[True][1]}
    # whole series without an external bound
    L, na = 256, 512
    A = torch.from_numpy(np.stack([synth.random_walk(L, 5000 + s) for s in range(na)]).astype(np.float32)).to(dev)
    api.pairwise(A[:64], A[:64], 26)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.pairwise(A, A, 26)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    band = L * (2 * 26 + 1) - 26 * 27
    out["pairwise"] = {"config": f"{na} x {na} random walks of {L} points, z-normalised, w=26",
                       "s": round(tp, 4), "pairs_per_s": na * na / tp, "band_cells_per_s": na * na * band / tp}
    ntr, nte = 4096, 256
    train = torch.from_numpy(np.stack([synth.random_walk(L, 20000 + s) for s in range(ntr)]).astype(np.float32)).to(dev)
    test = torch.from_numpy(np.stack([synth.random_walk(L, 90000 + s) for s in range(nte)]).astype(np.float32)).to(dev)
    api.nearest_series(train[:256], test[:16], 26, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.nearest_series(train, test, 26, 1)
    torch.cuda.synchronize()
    tn = time.perf_counter() - t0
    out["nn1_classification"] = {"config": f"{nte} test x {ntr} training random walks of {L} points, w=26, k=1",
                                 "s": round(tn, 4), "test_series_per_s": nte / tn,
                                 "pairs_per_s": nte * ntr / tn}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        cpu_baseline()
    vals, secs = [], []
    for _ in range(args.steps):
        cb = cpu_baseline()
        vals.append(cb["value"])
        secs.append(cb["seconds"])
    v = statistics.mean(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "windows/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.n), "n": args.n, "m": M, "queries": len(QUERY_SEEDS),
                       "w": [w for w, _ in SEARCHES], "k": 1, "parallelism": "host cores of rank 0",
                       "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "windows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT, help="reference length (default 2e7)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="all", choices=["all", "cascade", "nolb"],
                    help="searches per step (profiling aid; the benchmark is 'all')")
    ap.add_argument("--queries", default="1,2,3,4",
                    help="query seeds of the step (profiling aid; the benchmark is all four)")
    ap.add_argument("--batch-queries", type=int, default=32,
                    help="queries sampled from the batched mix (the first of each stratum and kind, against 8 "
                         "references); 0 skips it")
    ap.add_argument("--batch-strata", default="",
                    help="indices into the sampled strata to run alone (profiling aid; the benchmark runs all)")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the saturated and plain serving runs; 0 skips serving")
    ap.add_argument("--serve-poisson-requests", type=int, default=12, help="requests per Poisson rate")
    ap.add_argument("--serve-active", type=int, default=16, help="state slots of the serving loop")
    ap.add_argument("--serve-n", type=int, default=SERVE_N, help="serving reference length")
    ap.add_argument("--no-extensions", action="store_true", help="skip the extensions object")
    args = ap.parse_args()
    global SEARCHES, QUERY_SEEDS
    QUERY_SEEDS = tuple(int(x) for x in args.queries.split(","))
    if args.mode == "cascade":
        SEARCHES = [SEARCHES[0]]
    elif args.mode == "nolb":
        SEARCHES = [SEARCHES[1]]
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier()
    from paper_2010_05371_gb300 import api, synth

    n = args.n
    nw = n - M + 1
    R_np = synth.random_walk(n, 0).astype(np.float32)
    Qs_np = [synth.random_walk(M, s).astype(np.float32) for s in QUERY_SEEDS]
    R = torch.from_numpy(R_np).to(dev)
    Qs = [torch.from_numpy(q).to(dev) for q in Qs_np]
    stream = torch.cuda.current_stream(dev)

    from paper_2010_05371_gb300 import shard

    def step(Rd, Qd):
        # one rank: the whole search; N ranks: each rank searches its window
        # range (with the lQ - 1 halo) and the ranks merge their results
        out = []
        for (w, nolb) in SEARCHES:
            for q, seed in zip(Qd, QUERY_SEEDS):
                if world == 1:
                    idx, dist_, cnt = api.subseq_search(q, Rd, w, 1, no_lb=nolb, return_counters=True,
                                                        stream=stream)
                else:
                    holder = {}

                    def part(Qp, Rp, ww, kk, holder=holder, nolb=nolb):
                        i_, d_, c_ = api.subseq_search(Qp, Rp, ww, kk, no_lb=nolb, return_counters=True,
                                                       stream=stream)
                        holder["c"] = c_
                        return i_, d_

                    gi, gd = shard.sharded_search(part, q, Rd, w, 1, rank, world, device=dev)
                    idx, dist_ = torch.from_numpy(gi), torch.from_numpy(gd)
                    cnt = holder.get("c", {k_: 0 for k_ in api.COUNTER_NAMES})
                out.append((seed, w, nolb, idx, dist_, cnt))
        return out

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    for _ in range(args.warmup):
        step(R, Qs)
    torch.cuda.synchronize()

    gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
    gpu_id = gpu_uuid if gpu_uuid.startswith("GPU-") else f"GPU-{gpu_uuid}"
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms = []
    results = None
    main_ns = wider_ns = cells = launches = 0
    # per kind of search (nolb: the unconstrained searches without lower
    # bounds, whose first level is the dominant kernel; cascade: w = 103 with
    # the lower bounds): kernel ns, executed cells, searches
    per_kind = {True: [0, 0, 0], False: [0, 0, 0]}
    with ClockSampler(gpu_id) as clocks:
        barrier()
        torch.cuda.synchronize()
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()          # L2 flushed between steps (outside the timed events)
            ev0.record(stream)
            results = step(R, Qs)
            ev1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            for r in results:
                c = r[5]
                main_ns += c["ns_main"]
                wider_ns += c["ns_wider"]
                cells += c["cells"]
                launches += c["launches"]
                pk = per_kind[bool(r[2])]
                pk[0] += c["ns_main"] + c["ns_wider"]
                pk[1] += c["cells"]
                pk[2] += 1
        torch.cuda.synchronize()
        barrier()
        t_wall = time.perf_counter() - t_wall0
        # the DP cell's throughput ceiling, under the same clock record
        peak_rates = {m: api.cell_peak(m, PEAK_STEPS)[0] for m in PEAK_MODES}
        peak_rates["best"] = max(peak_rates.values())
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    # every window of every search is processed once, by one rank
    value = job_rate(len(SEARCHES) * len(QUERY_SEEDS) * nw, ms)

    # ---- end to end: the host-buffer entry point (subseq_search_host) on
    # pinned host arrays; every call copies its R and Q in and its result out ----
    R_pin = torch.from_numpy(R_np).pin_memory().numpy()
    Q_pin = [torch.from_numpy(q).pin_memory().numpy() for q in Qs_np]
    e2e_ms = []
    host = []
    for it in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if world == 1:
            host = [api.subseq_search_host(qh, R_pin, w, 1, no_lb=nolb)
                    for (w, nolb) in SEARCHES for qh in Q_pin]
        else:   # each rank copies in its slice only
            host = [shard.sharded_search(lambda Qp, Rp, ww, kk, nolb=nolb: api.subseq_search_host(Qp, Rp, ww, kk, no_lb=nolb),
                                         qh, R_pin, w, 1, rank, world, device=dev)
                    for (w, nolb) in SEARCHES for qh in Q_pin]
        if it > 0:  # first iteration warms the host path's scratch
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step_ms = max_over_ranks(statistics.mean(e2e_ms), world, dev)
    e2e = {"value": job_rate(len(SEARCHES) * len(QUERY_SEEDS) * nw, e2e_step_ms),
           "unit": "windows/s",
           "h2d_bytes_per_step": len(host) * (4 * (shard.slice_bounds(*shard.window_ranges(nw, world)[rank], M)[1]
                                                   - shard.slice_bounds(*shard.window_ranges(nw, world)[rank], M)[0])
                                              + 4 * M),
           "d2h_bytes_per_step": 16 * len(host), "ms_per_step": e2e_step_ms,
           "api": "subseq_search_host, one call per search, pinned host buffers"}

    # ---- roofline of the dominant kernel (search kernel, first level) ----
    nsearch = args.steps * len(results)
    clk = clocks.summary()
    golden = load_golden(n)

    def alg_of(kind):
        if not golden:
            return None
        return args.steps * sum(golden[(r[0], r[1], not r[2])]["audit_counters"]["cells"]
                                for r in results if bool(r[2]) == kind)

    peak = peak_rates["best"] / 1e12

    def roof_of(kind, kernel, traffic):
        ns, ex, ns_count = per_kind[kind]
        if ns <= 0:
            return None
        alg = alg_of(kind)
        used = alg if alg is not None else ex
        achieved = used / (ns / 1e9) / 1e12
        executed = ex / (ns / 1e9) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tcells/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                "kernel_ms_per_search": ns / 1e6 / ns_count,
                "work": ("algorithmic cells (oracle audit-mode EAPrunedDTW count at ub = NN distance)"
                         if alg is not None else "executed cells (no oracle count available)"),
                "executed_cells_achieved": executed, "executed_cells_frac": executed / peak,
                "executed_over_algorithmic": (ex / alg) if alg else None,
                "peak_basis": ("measured: eapdtw_cell_peak, the DP cell alone on every SM (CUDA events, "
                               "fastest of 3 launches), the fastest of its modes"),
                "peak_modes_tcells": {str(k): v / 1e12 for k, v in peak_rates.items() if k != "best"}}

    # the dominant kernel: the unconstrained searches' levels (the elastic
    # first level and its re-runs), timed with CUDA events inside the library
    roof = None if world > 1 else roof_of(True, "search_elastic_kernel (EAPrunedDTW elastic wavefront, unconstrained first level) "
                         "with its wider re-run levels", TRAFFIC_BYTES_PER_SEARCH)
    # the cascade searches (LB_Kim / LB_Keogh terms and banded DP cells; only
    # the DP cells are counted as work here)
    roof_cascade = None if world > 1 else roof_of(False, "search_kernel (LB cascade + banded EAPrunedDTW wavefront), all levels", None)
    alg_cells = None
    if golden:
        alg_cells = (alg_of(True) or 0) + (alg_of(False) or 0)

    # parity of this run's answers against the oracle's full-size results: the
    # distance within the tolerance of the oracle's; the index the oracle's, or
    # one whose oracle distance (from the stored top list) is within the same
    # tolerance of the oracle's best
    parity = None
    if golden:
        ok = 0
        for r in results:
            g = golden[(r[0], r[1], not r[2])]
            d, i = float(r[4].cpu()[0]), int(r[3].cpu()[0])
            tol = 1e-4 * max(g["nn_dist"], 1e-6 * M)
            top = {int(ti): float(td) for ti, td in g.get("top", [])}
            idx_ok = i == g["nn_index"] or (i in top and abs(top[i] - g["nn_dist"]) <= tol)
            if idx_ok and abs(d - g["nn_dist"]) <= tol:
                ok += 1
        parity = f"{ok}/{len(results)} searches match the oracle's nearest neighbour"

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    batched = serving = extensions = None
    if rank == 0 and world == 1 and not args.no_extensions:
        extensions = extensions_section(args, dev, R, Qs)
    if rank == 0 and world == 1:
        del flush
        torch.cuda.empty_cache()
        if args.batch_queries > 0:
            batched = batched_section(args, dev)
        if args.serve_requests > 0:
            serving = serving_section(args, dev)

    if rank == 0:
        per_mode = {}
        for r in results:
            key = f"w={r[1]}{' nolb' if r[2] else ' cascade'}"
            per_mode.setdefault(key, []).append(r[5]["ns_total"] / 1e6)
        line = {
            "metric": METRIC, "value": value, "unit": "windows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(n), "n": n, "m": M, "queries": len(QUERY_SEEDS),
                       "w": [w for w, _ in SEARCHES], "k": 1,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "parallelism": (f"window-range sharding over {world} ranks, merged by all-reduce MIN"
                                       if world > 1 else "1 GPU")},
            "dtw_cells_per_s": world * cells / args.steps / (ms / 1e3),
            "algorithmic_cells_per_s": (world * alg_cells / args.steps / (ms / 1e3)) if alg_cells else None,
            "queries_per_s": world * len(results) / (ms / 1e3),
            "search_ms": {k: round(statistics.mean(v), 3) for k, v in per_mode.items()},
            "roofline": roof,
            "roofline_cascade": roof_cascade,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "parity": parity,
            "batched": batched,
            "serving": serving,
            "extensions": extensions,
            "wall_s": round(t_wall, 3),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
