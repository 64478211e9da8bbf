"""Oracle results for the ECG-like large configuration, written to
tests/golden/ecg_large_oracle.json.

Workload: an ECG-like beat train of 20,000,000 points (seed 0, stored as
FP32; synth.ecg_like), queries of 256 and 512 points cut from a separate beat
train plus noise (synth.ecg_query, seeds 1 and 2), windows 5%, 20% and 50% of
the query length (w = ceil(ratio m): 13 / 52 / 128 and 26 / 103 / 256); every
search with the LB_Kim -> LB_Keogh EQ -> EC -> EAPrunedDTW cascade, k = 1.
For every search it records the nearest window (index, FP64 distance) of the
oracle's cascade search.  It calls nothing but oracle/ and the seeded
generators.

    python -m oracle.ecg_reference [--threads 8] [--n 20000000]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import oracle as O
from paper_2010_05371_gb300 import synth

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                   "ecg_large_oracle.json")

SEARCHES = [(qseed, m, math.ceil(r * m)) for qseed, m in ((1, 256), (2, 512)) for r in (0.05, 0.20, 0.50)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 8)
    ap.add_argument("--n", type=int, default=20_000_000)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    R = synth.ecg_like(args.n, 0)
    res = {"workload": f"ECG-like beat train n={args.n} seed 0; queries: ecg_query m=256 seed 1, m=512 seed 2",
           "generator": "paper_2010_05371_gb300.synth (numpy default_rng), rounded to FP32",
           "searches": []}
    for qseed, m, w in SEARCHES:
        Q = synth.ecg_query(m, qseed)
        t0 = time.time()
        idx, dist, cnt = O.search_cascade(Q, R, w, 1, use_lb=True, nthreads=args.threads)
        entry = {"query_seed": qseed, "m": m, "w": w, "nn_index": int(idx[0]), "nn_dist": float(dist[0]),
                 "oracle_seconds": round(time.time() - t0, 1)}
        res["searches"].append(entry)
        print(json.dumps(entry), flush=True)
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
