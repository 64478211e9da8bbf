"""The oracle against its pins, and planted mistakes that the pins must catch."""
import math

import numpy as np
import pytest

import oracle as O
import pins


@pytest.mark.parametrize("check", pins.ALL, ids=lambda c: c.__name__)
def test_pin(check):
    assert check() == []


# Each entry plants one plausible mistake in a copy of oracle.c: (name, text, replacement).
MUTANTS = [
    # Algorithm 3 exactly as printed: stage 4 reuses the cost of the stage-3 column.
    ("stage4_as_printed",
     "double c = cost(li[i - 1], co[j - 1]);  /* READING: recomputed */",
     "double c = cost(li[i - 1], co[prev_pruning_point - 1]);"),
    ("strict_ub_in_stage1",
     "if (curr[j] <= ub) pruning_point = j + 1;\n            else next_start = next_start + 1;",
     "if (curr[j] < ub) pruning_point = j + 1;\n            else next_start = next_start + 1;"),
    ("eq5_drops_diagonal",
     "D[i * cols + j] = cost(S[i - 1], T[j - 1]) + min3(top, left, diag);",
     "D[i * cols + j] = cost(S[i - 1], T[j - 1]) + min2(top, left);"),
    ("band_off_by_one",
     "if (abs64(i - j) > w) {\n                D[i * cols + j]",
     "if (abs64(i - j) >= w + 1 + (w > 2)) {\n                D[i * cols + j]"),
    ("sample_std",
     "v /= (double)m;\n    if (!(v > 0.0)) {",
     "v /= (double)(m - 1);\n    if (!(v > 0.0)) {"),
    ("keogh_wrong_side",
     "if (x[i] > U[i]) s += cost(x[i], U[i]);",
     "if (x[i] > U[i]) s += cost(x[i], L[i]);"),
    ("tie_to_larger_index",
     "return d1 < d2 || (d1 == d2 && i1 < i2);",
     "return d1 < d2 || (d1 == d2 && i1 > i2);"),
    ("no_window_in_alg3",
     "if (next_start < lo) next_start = lo;",
     ""),
    ("reversed_column_alg1",
     "double c = cost(li[i - 1], co[j - 1]);\n            curr[j] = c + min3(curr[j - 1], prev[j], prev[j - 1]);\n        }\n    }\n    double r",
     "double c = cost(li[i - 1], co[l_co - j]);\n            curr[j] = c + min3(curr[j - 1], prev[j], prev[j - 1]);\n        }\n    }\n    double r"),
    ("kim_wrong_index",
     "return cost(zc[0], zq[0]) + cost(zc[m - 1], zq[m - 1]);",
     "return cost(zc[0], zq[0]) + cost(zc[m - 1], zq[m - 2]);"),
    ("collision_ignores_ub",
     "if (curr[j] <= ub) pruning_point = j + 1;\n                else goto abandon;",
     "pruning_point = j + 1;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, tmp_path):
    src = O.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    so = O.compile_variant(src.replace(old, new), str(tmp_path))
    with O.use_library(so):
        fails = pins.all_checks(quick=True)
    assert fails, f"planted mistake {name} was not caught by any pin"


def test_eapruned_trace_invariants():
    """Algorithm 3 never computes more cells than the band holds, and next_start
    only moves right (Section 3: discard points extend the left border)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        m = int(rng.integers(5, 60))
        w = int(rng.integers(0, m))
        S, T = rng.standard_normal(m), rng.standard_normal(m)
        d = O.dtw(S, T, w)
        ub = d * rng.uniform(0.5, 1.5)
        v, tr = O.eapruned_dtw(S, T, w, ub, trace=True)
        band = sum(1 for i in range(1, m + 1) for j in range(1, m + 1) if abs(i - j) <= w)
        assert tr["cells"] <= band
        assert np.all(np.diff(tr["next_start"]) >= 0)
        assert (v == d) == (d <= ub)
