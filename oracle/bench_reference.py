"""Oracle results for the large benchmark workload, written to
tests/golden/bench_large_oracle.json.

Workload (the "large" configuration of the benchmark): a Gaussian random walk
of 20,000,000 points (seed 0, stored as FP32), four random-walk queries of
length 1024 (seeds 1-4); each query is searched with w = 103 (10%, LB_Kim ->
LB_Keogh EQ -> EC -> EAPrunedDTW) and with w = 1024 (unconstrained, no lower
bounds).  For every search this script records, from the oracle only:
  - the nearest window (index, distance) of the FP64 cascade search;
  - the EAPrunedDTW cells of an audit-mode search whose ub is fixed at that
    distance (the work the method itself must do; order-independent);
  - with --add-top K (run on an existing file), the K nearest windows of the
    FP64 search, so that a GPU answer at another index can be checked for tie
    equivalence against the oracle's own distance at that index.
It calls nothing but oracle/ and the seeded generators; it takes tens of
minutes on 8 cores.

    python -m oracle.bench_reference [--threads 8] [--n 20000000]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

import oracle as O
from paper_2010_05371_gb300 import synth

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                   "bench_large_oracle.json")

SEARCHES = [  # (query seed, w, use_lb)
    (1, 103, True), (2, 103, True), (3, 103, True), (4, 103, True),
    (1, 1024, False), (2, 1024, False), (3, 1024, False), (4, 1024, False),
]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 8)
    ap.add_argument("--n", type=int, default=20_000_000)
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--add-top", type=int, default=0,
                    help="add the K nearest windows of every search to an existing file")
    args = ap.parse_args()
    R = synth.random_walk(args.n, 0)
    if args.add_top:
        with open(args.out) as f:
            res = json.load(f)
        for entry in res["searches"]:
            Q = synth.random_walk(entry["m"], entry["query_seed"])
            idx, dist, _ = O.search_cascade(Q, R, entry["w"], args.add_top, use_lb=True, nthreads=args.threads)
            entry["top"] = [[int(i), float(d)] for i, d in zip(idx, dist)]
            print(json.dumps({"query_seed": entry["query_seed"], "w": entry["w"], "top": entry["top"]}), flush=True)
            with open(args.out, "w") as f:
                json.dump(res, f, indent=1)
        return
    res = {"workload": f"random walk n={args.n} seed 0; queries: random walks m=1024 seeds 1-4",
           "generator": "numpy default_rng(seed), cumsum of standard normals, rounded to FP32",
           "searches": []}
    for qseed, w, use_lb in SEARCHES:
        Q = synth.random_walk(1024, qseed)
        t0 = time.time()
        # the nearest neighbour (the cascade with lower bounds is the fastest exact oracle search)
        idx, dist, cnt = O.search_cascade(Q, R, w, 1, use_lb=True, nthreads=args.threads)
        t1 = time.time()
        _, _, audit = O.search_cascade(Q, R, w, 1, use_lb=use_lb, ub_fixed=float(dist[0]),
                                       nthreads=args.threads)
        t2 = time.time()
        entry = {"query_seed": qseed, "m": 1024, "w": w, "lower_bounds": use_lb,
                 "nn_index": int(idx[0]), "nn_dist": float(dist[0]),
                 "audit_counters": audit, "oracle_seconds": [round(t1 - t0, 1), round(t2 - t1, 1)]}
        res["searches"].append(entry)
        print(json.dumps(entry), flush=True)
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
