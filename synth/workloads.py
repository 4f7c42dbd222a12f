"""Seeded synthetic workloads: protocol batches, spheroid sizes, surrogate features.

Inputs only: nothing here computes any part of the simulation.  Both the CUDA
library and the FP64 oracle are fed from these generators.

Protocols are lists of (dose Gy, wait h) pairs whose first wait counts from
t = 0, as the paper defines them ("Defining the search problem").  Waits sit
on the paper's 30-minute grid.  A protocol whose total dose exceeds the cap is
repaired with the paper's dose guard (GA details, "Crossover"): subtract one
dose step from the currently largest dose (earliest on ties) until the total
is within the cap.
"""
from __future__ import annotations

import math

import numpy as np

WAITS_6_TO_60 = tuple(float(w) for w in range(6, 61, 6))  # {6, 12, ..., 60} h


def cap_total_dose(doses, cap: float, step: float) -> list:
    d = [float(x) for x in doses]
    while sum(d) > cap + 1e-9:
        j = int(np.argmax(d))  # argmax returns the earliest maximum
        d[j] = max(0.0, d[j] - step)
    return d


def daily_fractions(n: int = 10, dose: float = 2.0, interval_h: float = 24.0):
    """n x dose Gy at t = 0, interval, 2 interval, ...: ([doses], [waits])."""
    return [dose] * n, [0.0] + [interval_h] * (n - 1)


def benchmark_bmi():
    """BMI of the paper: 8 x 1.25 Gy with 6 h / 18 h alternating waits."""
    return [1.25] * 8, [0.0, 6, 18, 6, 18, 6, 18, 6]


def benchmark_bmii():
    """BMII of the paper: 5 x 2 Gy, one per day."""
    return [2.0] * 5, [0.0, 24, 24, 24, 24]


def ga_batch(n: int = 256, seed: int = 2, n_frac: int = 10, doses=(0.5, 1.0, 1.5, 2.0, 2.5),
             waits=WAITS_6_TO_60, cap: float = 20.0, dose_step: float = 0.5):
    """Uniform GA population: each protocol has n_frac fractions, dose and wait
    drawn uniformly per fraction from the given sets, total capped by the guard."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        d = rng.choice(doses, size=n_frac).tolist()
        w = rng.choice(waits, size=n_frac).tolist()
        out.append((cap_total_dose(d, cap, dose_step), [float(x) for x in w]))
    return out


def lattice_for_radius(R: int) -> int:
    """Lattice side 2.5 x the spheroid diameter, rounded up to a multiple of 16."""
    return 16 * math.ceil(5 * R / 16)


def ragged_batch(n: int = 1024, seed: int = 3, r_min: int = 4, r_max: int = 20, f_min: int = 5, f_max: int = 15,
                 doses=(1.0, 2.0, 3.0, 4.0, 5.0), waits=WAITS_6_TO_60, cap: float = 30.0, dose_step: float = 1.0):
    """Hypofractionated ragged batch: radius uniform in [r_min, r_max], lattice
    from the radius, fraction count uniform in [f_min, f_max]."""
    rng = np.random.default_rng(seed)
    R = rng.integers(r_min, r_max + 1, size=n)
    L = np.array([lattice_for_radius(int(r)) for r in R], dtype=np.int32)
    protos = []
    for _ in range(n):
        k = int(rng.integers(f_min, f_max + 1))
        d = rng.choice(doses, size=k).tolist()
        w = rng.choice(waits, size=k).tolist()
        protos.append((cap_total_dose(d, cap, dose_step), [float(x) for x in w]))
    return L, R.astype(np.int32), protos
