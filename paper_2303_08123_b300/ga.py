"""Thin host GA over radiotherapy protocols (arxiv 2303.08123, "The Genetic
Algorithm (GA)" and the GA operator details).

A genotype is the paper's sparse dose vector: entry i is the dose (Gy) given
i * 30 min after the start, zero for no fraction ("Protocol Representation").
Doses sit on a 0.25 Gy grid up to d_max, fractions are at least `min_gap`
slots apart and the total dose is capped ("GA Resolution, constraints").

Operators (GA operator details):
  selection   simple (top fraction), roulette (p_i = f_i / sum f), tournament
              (rank-based, probability q (1 - q)^(k - 1) for the k-th best)
  elitism     the best 10 % pass unchanged
  crossover   single point (cut in 25-75 % of the length), two points (25-50 %,
              50-75 %), uniform (per gene, complementary children)
  mutation    swap, split, dose-time, dose-value
  guards      relocate doses that violate the minimum interval (skip when no
              room), then remove 0.25 Gy from the currently largest dose until
              the total is within the cap

Fitness comes from the batched simulator (or, when screening, first from the
surrogate).  Everything here is host bookkeeping on small arrays.
"""
from __future__ import annotations

import dataclasses

import numpy as np

DOSE_STEP = 0.25
SLOT_H = 0.5


@dataclasses.dataclass
class GAConfig:
    n_slots: int = 240          # 5 days at 30 min
    d_max: float = 2.0          # largest single fraction (Gy)
    total_cap: float = 10.0     # total dose (Gy)
    min_gap: int = 12           # minimum slots between fractions (6 h)
    population: int = 40
    elite_frac: float = 0.10
    parent_frac: float = 0.40
    selection: str = "simple"   # simple | roulette | tournament
    crossover: str = "two_point"  # single_point | two_point | uniform
    mutations: tuple = ("swap", "split", "dose_time")
    p_mut: float = 0.3
    tournament_k: int = 16
    tournament_q: float = 0.9


# ----------------------------------------------------------------------------- encoding
def to_pairs(vec):
    """Sparse dose vector -> ([doses], [waits in h]); the first wait counts from t = 0."""
    idx = np.flatnonzero(np.asarray(vec) > 0)
    doses = [float(vec[i]) for i in idx]
    waits, prev = [], 0
    for i in idx:
        waits.append((i - prev) * SLOT_H)
        prev = i
    return doses, waits


def from_pairs(doses, waits, n_slots):
    vec = np.zeros(n_slots)
    t = 0.0
    for d, w in zip(doses, waits):
        t += w
        i = int(round(t / SLOT_H))
        if i >= n_slots:
            raise ValueError("protocol longer than the vector")
        vec[i] += d
    return vec


# ----------------------------------------------------------------------------- guards
def guard_interval(vec, cfg: GAConfig, rng):
    """Move doses that sit closer than min_gap slots to an earlier dose to a
    random slot that respects the interval; drop the move (keep the dose where
    it is merged into its neighbour) when no slot is free."""
    vec = np.asarray(vec, dtype=float).copy()
    while True:
        idx = np.flatnonzero(vec > 0)
        bad = [j for a, j in zip(idx[:-1], idx[1:]) if j - a < cfg.min_gap]
        if not bad:
            return vec
        j = bad[0]
        d = vec[j]
        vec[j] = 0.0
        occupied = np.flatnonzero(vec > 0)
        free = [s for s in range(cfg.n_slots) if np.all(np.abs(occupied - s) >= cfg.min_gap)]
        if free:
            vec[free[rng.integers(len(free))]] = d
        else:  # no room: the paper skips the allocation; fold the dose into the previous fraction
            prev = occupied[occupied < j]
            k = prev[-1] if len(prev) else occupied[0]
            vec[k] = min(cfg.d_max, vec[k] + d)


def guard_total(vec, cfg: GAConfig):
    """Subtract 0.25 Gy from the currently largest dose (earliest on ties)
    until the total is within the cap."""
    vec = np.asarray(vec, dtype=float).copy()
    while vec.sum() > cfg.total_cap + 1e-9:
        j = int(np.argmax(vec))
        vec[j] = max(0.0, vec[j] - DOSE_STEP)
    return vec


def repair(vec, cfg: GAConfig, rng):
    vec = np.clip(np.round(np.asarray(vec, dtype=float) / DOSE_STEP) * DOSE_STEP, 0.0, cfg.d_max)
    return guard_total(guard_interval(vec, cfg, rng), cfg)


def random_protocol(cfg: GAConfig, rng, n_frac=None):
    vec = np.zeros(cfg.n_slots)
    n_frac = n_frac or int(rng.integers(1, cfg.n_slots // cfg.min_gap + 1))
    for _ in range(n_frac):
        vec[rng.integers(cfg.n_slots)] += DOSE_STEP * rng.integers(1, int(cfg.d_max / DOSE_STEP) + 1)
    return repair(vec, cfg, rng)


# ----------------------------------------------------------------------------- selection
def select_simple(fit, n):
    return list(np.argsort(-np.asarray(fit), kind="stable")[:n])


def select_roulette(fit, n, rng):
    f = np.asarray(fit, dtype=float)
    f = f - min(0.0, f.min())  # probabilities need non-negative fitness
    p = f / f.sum() if f.sum() > 0 else np.full(len(f), 1.0 / len(f))
    cum = np.cumsum(p)
    return [int(np.searchsorted(cum, rng.random() * cum[-1], side="left")) for _ in range(n)]


def select_tournament(fit, n, rng, k=16, q=0.9):
    order = np.argsort(-np.asarray(fit), kind="stable")
    out = []
    for _ in range(n):
        entrants = np.sort(rng.choice(len(order), size=min(k, len(order)), replace=False))
        # rank r (0 = best) among the entrants wins with probability q (1 - q)^r
        r = 0
        while r < len(entrants) - 1 and rng.random() >= q:
            r += 1
        out.append(int(order[entrants[r]]))
    return out


# ----------------------------------------------------------------------------- crossover
def crossover(a, b, kind, rng):
    n = len(a)
    if kind == "single_point":
        c = int(rng.integers(int(0.25 * n), int(0.75 * n) + 1))
        return np.concatenate([a[:c], b[c:]]), np.concatenate([b[:c], a[c:]])
    if kind == "two_point":
        c1 = int(rng.integers(int(0.25 * n), int(0.50 * n) + 1))
        c2 = int(rng.integers(int(0.50 * n), int(0.75 * n) + 1))
        return (np.concatenate([a[:c1], b[c1:c2], a[c2:]]), np.concatenate([b[:c1], a[c1:c2], b[c2:]]))
    if kind == "uniform":
        m = rng.random(n) < 0.5
        return np.where(m, a, b), np.where(m, b, a)
    raise ValueError(kind)


# ----------------------------------------------------------------------------- mutation
def mutate(vec, cfg: GAConfig, rng):
    vec = np.asarray(vec, dtype=float).copy()
    for kind in cfg.mutations:
        if rng.random() >= cfg.p_mut:
            continue
        idx = np.flatnonzero(vec > 0)
        if kind == "swap" and len(idx):  # a dose trades places with a random slot
            i, j = int(rng.choice(idx)), int(rng.integers(cfg.n_slots))
            vec[i], vec[j] = vec[j], vec[i]
        elif kind == "split":  # a dose > 0.25 Gy becomes two parts at random slots, each within d_max
            big = idx[vec[idx] > DOSE_STEP]
            if len(big):
                i = int(rng.choice(big))
                part = DOSE_STEP * rng.integers(1, int(round(vec[i] / DOSE_STEP)))
                rest = vec[i] - part
                vec[i] = 0.0
                for d in (part, rest):
                    for _ in range(8):  # look for a slot that stays within d_max
                        j = int(rng.integers(cfg.n_slots))
                        if vec[j] + d <= cfg.d_max + 1e-9:
                            vec[j] += d
                            break
                    else:
                        vec[i] += d
        elif kind == "dose_time" and len(idx):  # move a dose, clamp at d_max, remainder stays
            i, j = int(rng.choice(idx)), int(rng.integers(cfg.n_slots))
            moved = min(vec[i], cfg.d_max - vec[j]) if j != i else 0.0
            moved = max(0.0, np.floor(moved / DOSE_STEP) * DOSE_STEP)
            vec[j] += moved
            vec[i] -= moved
        elif kind == "dose_value" and len(idx):  # raise a dose using the slack under the cap
            slack = cfg.total_cap - vec.sum()
            if slack > 0:
                i = int(rng.choice(idx))
                room = min(slack, cfg.d_max - vec[i])
                steps = int(np.floor(room / DOSE_STEP + 1e-9))
                if steps > 0:
                    vec[i] += DOSE_STEP * rng.integers(1, steps + 1)
    return repair(vec, cfg, rng)


# ----------------------------------------------------------------------------- generation
def next_generation(pop, fit, cfg: GAConfig, rng, n_children=None):
    """Elites (simple selection) + children from selected parents by crossover
    then mutation ("The Main GA Loop")."""
    n = len(pop)
    n_elite = max(1, int(round(cfg.elite_frac * n)))
    n_par = max(2, int(round(cfg.parent_frac * n)))
    n_children = n - n_elite if n_children is None else n_children
    elites = [pop[i].copy() for i in select_simple(fit, n_elite)]
    if cfg.selection == "simple":
        parents = select_simple(fit, n_par)
    elif cfg.selection == "roulette":
        parents = select_roulette(fit, n_par, rng)
    else:
        parents = select_tournament(fit, n_par, rng, cfg.tournament_k, cfg.tournament_q)
    children = []
    while len(children) < n_children:
        a, b = rng.choice(parents, size=2, replace=False) if len(set(parents)) > 1 else (parents[0], parents[0])
        for c in crossover(pop[a], pop[b], cfg.crossover, rng):
            if len(children) < n_children:
                children.append(mutate(c, cfg, rng))
    return elites, children


def is_valid(vec, cfg: GAConfig) -> bool:
    v = np.asarray(vec)
    idx = np.flatnonzero(v > 0)
    on_grid = np.allclose(np.round(v / DOSE_STEP) * DOSE_STEP, v)
    gaps = np.all(np.diff(idx) >= cfg.min_gap) if len(idx) > 1 else True
    return bool(on_grid and gaps and v.max(initial=0) <= cfg.d_max + 1e-9 and v.sum() <= cfg.total_cap + 1e-9)
