"""Oracle results for a seeded sample of the batched mix, written to
tests/golden/batched_mix_oracle.json.

The mix: 1,024 queries with lengths log-uniform in 64-2048 and window ratios
uniform in 0-1 (w = ceil(ratio m)), random walk or ECG-like by a coin flip,
k = 1 or 5 by a coin flip (query seed 2; query q's values from seed 1000 + q),
each against 8 random-walk references with lengths log-uniform in 1e5-1e7
(seed 3; reference j from seed 100 + j).  This script draws 64 (query,
reference) items at random (seed 7) among the items whose reference is one of
the four shortest, and records each item's k nearest windows from the
oracle's FP64 cascade search.  It calls nothing but oracle/ and the seeded
generators; it takes tens of minutes on 8 cores.

    python -m oracle.batched_reference [--threads 8]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

import oracle as O
from paper_2010_05371_gb300 import synth

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                   "batched_mix_oracle.json")
QUERIES, REFS, SAMPLE = 1024, 8, 64


def mix():
    """(reference lengths, [(m, w, ecg, k) per query]) of the batched mix."""
    rr = np.random.default_rng(3)
    lens = [int(round(math.exp(rr.uniform(math.log(1e5), math.log(1e7))))) for _ in range(REFS)]
    rq = np.random.default_rng(2)
    qs = []
    for _ in range(QUERIES):
        m = int(round(math.exp(rq.uniform(math.log(64), math.log(2048)))))
        w = int(math.ceil(rq.uniform(0.0, 1.0) * m))
        ecg = bool(rq.random() < 0.5)
        k = 1 if rq.random() < 0.5 else 5
        qs.append((m, w, ecg, k))
    return lens, qs


def sample_items(lens):
    short = sorted(range(REFS), key=lambda j: lens[j])[:4]
    rs = np.random.default_rng(7)
    picks = set()
    while len(picks) < SAMPLE:
        picks.add((int(rs.integers(0, QUERIES)), int(short[rs.integers(0, len(short))])))
    return sorted(picks)


def query_values(q, m, ecg):
    return synth.ecg_query(m, 1000 + q) if ecg else synth.random_walk(m, 1000 + q)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 8)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    lens, qs = mix()
    refs = {}
    res = {"mix": "1024 queries (seed 2, values seed 1000+q) x 8 references (seed 3, values seed 100+j); "
                  "64 items drawn with seed 7 among the 4 shortest references",
           "items": []}
    for q, j in sample_items(lens):
        m, w, ecg, k = qs[q]
        if j not in refs:
            refs[j] = synth.random_walk(lens[j], 100 + j)
        Q = query_values(q, m, ecg)
        t0 = time.time()
        idx, dist, _ = O.search_cascade(Q, refs[j], w, k, use_lb=True, nthreads=args.threads)
        e = {"query": q, "ref": j, "m": m, "w": w, "ecg": ecg, "k": k, "n": lens[j],
             "idx": [int(x) for x in idx], "dist": [float(x) for x in dist], "oracle_seconds": round(time.time() - t0, 1)}
        res["items"].append(e)
        print(json.dumps(e), flush=True)
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
