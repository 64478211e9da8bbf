"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module generates data only: it holds none of the search arithmetic
(no normalisation, no bounds, no DTW).  All generators use numpy's
``default_rng(seed)`` (PCG64) so that every run of every side sees the same
series.  Series are returned as float64 arrays holding FP32-representable
values (``astype(float32).astype(float64)``): the device stores FP32 and the
oracle reads exactly the same numbers in FP64.

Workload shapes follow the experiments of Section 5 of the paper (query
lengths 128-1024, window ratios 0.1-0.5, long references); the paper's
datasets are not available, so random walks and an ECG-like beat train stand
in for them.
"""
from __future__ import annotations

import math

import numpy as np


def f32(x: np.ndarray) -> np.ndarray:
    """Round to FP32 and return as float64 (the values both sides use)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def random_walk(n: int, seed: int) -> np.ndarray:
    """Gaussian random walk: x_t = sum_{s<=t} e_s, e_s ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    return f32(np.cumsum(rng.standard_normal(n)))


# ECG-like beat: five Gaussian bumps (P, Q, R, S, T waves) at fixed phase
# positions of the beat, widths as a fraction of the beat period, and signs.
_BUMP_POS = (0.15, 0.35, 0.40, 0.45, 0.70)
_BUMP_WIDTH = (0.035, 0.012, 0.010, 0.012, 0.050)
_BUMP_SIGN = (1.0, -1.0, 1.0, -1.0, 1.0)


def ecg_like(n: int, seed: int, period=(200, 300), noise: float = 0.05,
             drift_amp: float = 0.3, drift_period=(5e3, 5e4)) -> np.ndarray:
    """Quasi-periodic beat train of n points.

    Beat periods are uniform in ``period`` (jitter per beat); each beat is a
    sum of 5 Gaussian bumps with amplitudes uniform in [0.1, 1.5] and fixed
    signs; a slow sinusoidal baseline drift (amplitude ``drift_amp``, period
    uniform in ``drift_period``) and N(0, noise) are added.
    """
    rng = np.random.default_rng(seed)
    nbeats = int(math.ceil(n / period[0])) + 2
    periods = rng.uniform(period[0], period[1], size=nbeats)
    starts = np.concatenate([[0.0], np.cumsum(periods)[:-1]]) - rng.uniform(0, period[0])
    amps = rng.uniform(0.1, 1.5, size=(nbeats, 5))
    t = np.arange(n, dtype=np.float64)
    beat = np.searchsorted(starts, t, side="right") - 1
    beat = np.clip(beat, 0, nbeats - 1)
    phase = (t - starts[beat]) / periods[beat]
    x = np.zeros(n, dtype=np.float64)
    for k in range(5):
        s = _BUMP_WIDTH[k]
        x += _BUMP_SIGN[k] * amps[beat, k] * np.exp(-0.5 * ((phase - _BUMP_POS[k]) / s) ** 2)
    pd = rng.uniform(drift_period[0], drift_period[1])
    x += drift_amp * np.sin(2.0 * np.pi * t / pd + rng.uniform(0, 2 * np.pi))
    x += rng.normal(0.0, noise, size=n)
    return f32(x)


def ecg_query(m: int, seed: int, noise: float = 0.1, train_len: int = 20000) -> np.ndarray:
    """A query of length m cut from a separate seeded beat train plus N(0, noise)."""
    rng = np.random.default_rng(seed)
    train = ecg_like(train_len, seed=seed + 1_000_003, noise=0.05)
    off = int(rng.integers(0, train_len - m))
    return f32(train[off:off + m] + rng.normal(0.0, noise, size=m))


def window_from_ratio(ratio: float, m: int) -> int:
    """Warping window from a ratio of the query length: w = ceil(ratio * m)."""
    return int(math.ceil(ratio * m - 1e-12))


def random_series(n: int, seed: int, lo: float = -3.0, hi: float = 3.0) -> np.ndarray:
    """Uniform noise (for small DTW pair tests)."""
    rng = np.random.default_rng(seed)
    return f32(rng.uniform(lo, hi, size=n))


def small_int_series(n: int, seed: int, lo: int = 0, hi: int = 5) -> np.ndarray:
    """Small integers (exact arithmetic, many ties) for brute-force checks."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=n).astype(np.float64)


def loguniform_int(rng: np.random.Generator, lo: float, hi: float, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size)).astype(np.int64)
