"""Tumour case library and the paper's multi-tumour fitness.

The paper scores a protocol on a library of ten 10-day-old tumours grown
untreated from a small seed in the replenished medium ("The tumour case
library"), several evaluations per tumour, and uses the mean of f = 1500 - n
over all of them ("The fitness function & experimental setup").  The published
library is not available; this module grows one with the same simulator (each
tumour from its own seeded spheroid, so they differ) and evaluates protocols on
it, every (protocol, tumour, replicate) triple in its own slot of one batch.
"""
from __future__ import annotations

import numpy as np

from .sim import Simulator, csr

STEPS_PER_HOUR = 600


def grow_library(n_tumours: int, L: int, seed_radius: int, grow_h: int, seed: int, **cfg) -> Simulator:
    """Grow n_tumours untreated spheroids for grow_h hours; returns the batch
    holding them (slot t = tumour t)."""
    lib = Simulator([L] * n_tumours, [seed_radius] * n_tumours, seed=seed, init_word=0xFFFFFFFE,
                    t_end_steps=grow_h * STEPS_PER_HOUR, **cfg)
    lib.load_protocols(*csr([([], [])] * n_tumours))
    lib.run(0)
    return lib


def evaluate(protocols, library: Simulator, replicates: int, seed: int, regrowth_h: int = 120,
             n_max: float = 1500.0, **cfg):
    """Mean and standard deviation of f = n_max - n per protocol over every
    library tumour x replicate, and the raw counts (protocol, tumour, replicate)."""
    T = library.n
    P = len(protocols)
    slots = [(p, t, r) for p in range(P) for t in range(T) for r in range(replicates)]
    L = [int(library.L[t]) for _, t, _ in slots]
    sim = Simulator(L, [-1] * len(slots), seed=seed, regrowth_h=regrowth_h, n_max_fitness=n_max, **cfg)
    sim.load_protocols(*csr([protocols[p] for p, _, _ in slots]))
    for k, (_, t, _) in enumerate(slots):
        sim.copy_lattice(k, library, t)
    sim.run(0)
    n, f = sim.fitness()
    sim.close()
    counts = n.reshape(P, T, replicates)
    fit = f.reshape(P, T * replicates)
    return fit.mean(axis=1), fit.std(axis=1), counts
