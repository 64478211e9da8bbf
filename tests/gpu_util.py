"""Helpers shared by the GPU parity tests."""
import math

import numpy as np

import oracle as O

REL_TOL = 1e-4  # relative distance tolerance (FP32 DP against the FP64 oracle)


def dist_close(got: float, ref: float, m: int) -> bool:
    if math.isinf(ref) or math.isinf(got):
        return math.isinf(ref) and math.isinf(got)
    return abs(got - ref) <= REL_TOL * max(ref, 1e-6 * m)


def check_topk(gi, gd, oi, od, Q, R, w):
    """k-NN parity: distances within tolerance position by position; an index
    that differs must be tie-equivalent (its oracle distance is within the
    tolerance of the oracle's distance at that rank)."""
    m = len(Q)
    gi, gd = [int(x) for x in gi], [float(x) for x in gd]
    zq = O.znorm(Q)
    for j, (a, b, c, d) in enumerate(zip(gi, gd, oi, od)):
        assert dist_close(b, d, m), f"rank {j}: gpu dist {b} vs oracle {d}"
        if a != c:
            assert a >= 0, f"rank {j}: gpu index {a} vs oracle {c}"
            rescored = O.dtw(O.znorm(R[a:a + m]), zq, w)
            assert dist_close(rescored, d, m), f"rank {j}: gpu index {a} (oracle dist {rescored}) vs {c} ({d})"
    assert len(set(x for x in gi if x >= 0)) == len([x for x in gi if x >= 0]), "duplicate indices"
