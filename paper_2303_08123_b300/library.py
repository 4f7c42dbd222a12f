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

# The paper's library: ten tumours, each grown untreated for 10 days from a
# seed of about 200 cells, every protocol scored over all of them with several
# evaluations each ("The tumour case library", "The fitness function &
# experimental setup").  This build's reading: a seed ball of radius 4 (257
# lattice sites, the ball closest to 200 cells from above), 240 h of growth
# on 48^3 lattices (the tumours stay well inside the faces), 8 replicate
# evaluations per (protocol, tumour).
PAPER_CASES, PAPER_SEED_RADIUS, PAPER_GROW_H, PAPER_L, PAPER_REPLICATES = 10, 4, 240, 48, 8


def grow_library(n_tumours: int, L: int, seed_radius: int, grow_h: int, seed: int, **cfg) -> Simulator:
    """Grow n_tumours untreated spheroids for grow_h hours; returns the batch
    holding them (slot t = tumour t)."""
    lib = Simulator([L] * n_tumours, [seed_radius] * n_tumours, seed=seed, init_word=0xFFFFFFFE,
                    t_end_steps=grow_h * STEPS_PER_HOUR, **cfg)
    lib.load_protocols(*csr([([], [])] * n_tumours))
    lib.run(0)
    return lib


def paper_library(seed: int, **cfg) -> Simulator:
    """The library in the paper's shape: PAPER_CASES tumours grown PAPER_GROW_H
    hours from seed balls of radius PAPER_SEED_RADIUS on PAPER_L^3 lattices."""
    return grow_library(PAPER_CASES, PAPER_L, PAPER_SEED_RADIUS, PAPER_GROW_H, seed, **cfg)


def evaluation_batch(protocols, library: Simulator, replicates: int, seed: int, regrowth_h: int = 120,
                     n_max: float = 1500.0, **cfg):
    """One batch holding every (protocol, tumour, replicate) triple in its own
    slot, each slot started from its tumour by a device-side copy.  Returns
    (batch, slots); replicates differ in the slot's Philox protocol word."""
    T = library.n
    slots = [(p, t, r) for p in range(len(protocols)) for t in range(T) for r in range(replicates)]
    L = [int(library.L[t]) for _, t, _ in slots]
    sim = Simulator(L, [-1] * len(slots), seed=seed, regrowth_h=regrowth_h, n_max_fitness=n_max, **cfg)
    sim.load_protocols(*csr([protocols[p] for p, _, _ in slots]))
    for k, (_, t, _) in enumerate(slots):
        sim.copy_lattice(k, library, t)
    return sim, slots


def evaluate(protocols, library: Simulator, replicates: int, seed: int, regrowth_h: int = 120,
             n_max: float = 1500.0, **cfg):
    """Mean and standard deviation of f = n_max - n per protocol over every
    library tumour x replicate, and the raw counts (protocol, tumour, replicate)."""
    T = library.n
    P = len(protocols)
    sim, _ = evaluation_batch(protocols, library, replicates, seed, regrowth_h, n_max, **cfg)
    sim.run(0)
    n, f = sim.fitness()
    sim.close()
    counts = n.reshape(P, T, replicates)
    fit = f.reshape(P, T * replicates)
    return fit.mean(axis=1), fit.std(axis=1), counts
