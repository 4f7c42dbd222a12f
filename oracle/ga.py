"""CPU oracle of one GA generation over dose vectors (arxiv 2303.08123, "The
Genetic Algorithm (GA)", "The Main GA Loop" and the GA operator details:
selection, elitism, crossover, mutation and the two guards).

TEST INFRASTRUCTURE ONLY: plain Python loops over numpy rows, slow and direct;
the tests compare the device GA (libga) with it byte for byte.  Shares no code
with the CUDA library; random numbers come from this package's own Philox
(oracle.c, pinned against an independent implementation in the tests).

A genotype is a row of S integer dose units, entry i = dose at i * 30 min
("Protocol Representation").  Each random decision takes one Philox4x32-10
draw: counter (k, generation, purpose, individual), k counting the draws of
that individual; u = (x0 >> 8) * 2^-24, pick(n) = ((x0 >> 8) * n) >> 24.
Purposes: 3 parent selection, 4 children, 5 initial population.

Parity status: pinned by tests/test_ga_oracle.py (validity of every output
under the guards, elites equal the best individuals, simple selection equals a
sort, a certain tournament (q = 1, k = P) returns the best, roulette
frequencies follow the fitness shares, crossover conserves the parents' genes
slot by slot, mutations conserve the total dose where the paper says they do).
"""
from __future__ import annotations

import ctypes
import dataclasses
import struct

import numpy as np

from . import lib, _key

PURPOSE_SELECT, PURPOSE_CHILD, PURPOSE_INIT = 3, 4, 5
SEL_SIMPLE, SEL_ROULETTE, SEL_TOURNAMENT = 0, 1, 2
X_SINGLE, X_TWO, X_UNIFORM = 0, 1, 2
MUT_SWAP, MUT_SPLIT, MUT_DOSE_TIME, MUT_DOSE_VALUE = 1, 2, 4, 8


@dataclasses.dataclass
class GAParams:
    n_slots: int = 240
    d_max: int = 8            # units (0.25 Gy each: 2 Gy)
    total_cap: int = 40       # units (10 Gy)
    min_gap: int = 12         # slots (6 h)
    n_elite: int = 4
    n_parents: int = 16
    selection: int = SEL_SIMPLE
    crossover: int = X_TWO
    mutations: int = MUT_SWAP | MUT_SPLIT | MUT_DOSE_TIME
    p_mut: float = 0.3
    tournament_k: int = 16
    tournament_q: float = 0.9


def f32(x: float) -> float:
    """Round to the nearest FP32 value (the precision the probability comparisons use)."""
    return struct.unpack("f", struct.pack("f", x))[0]


class Draws:
    """The draw sequence of one individual in one generation."""

    def __init__(self, seed: int, who: int, gen: int, purpose: int):
        self.key = _key(seed)
        self.ctr = np.array([0, gen, purpose, who], dtype=np.uint32)
        self.out = np.empty(4, dtype=np.uint32)
        self.k = 0

    def word(self) -> int:
        self.ctr[0] = self.k
        self.k += 1
        P = ctypes.POINTER(ctypes.c_uint32)
        lib().or_philox4x32_10(self.ctr.ctypes.data_as(P), self.key.ctypes.data_as(P), self.out.ctypes.data_as(P))
        return int(self.out[0])

    def u(self) -> float:
        return (self.word() >> 8) * 2.0 ** -24

    def pick(self, n: int) -> int:
        return ((self.word() >> 8) * n) >> 24


# ----------------------------------------------------------------------------- ranking
def fitness_key(f: float) -> int:
    """Total order on FP32 fitness: larger is fitter, NaN least fit."""
    f = np.float32(f)
    if np.isnan(f):
        return 0
    b = int(np.array(f, dtype=np.float32).view(np.uint32))
    return (~b) & 0xFFFFFFFF if b & 0x80000000 else b | 0x80000000


def ranking(fit) -> list:
    """Indices from the fittest down; ties go to the lower index."""
    keys = [fitness_key(f) for f in fit]
    return sorted(range(len(fit)), key=lambda i: (-keys[i], i))


# ----------------------------------------------------------------------------- selection
def select_parents(fit, order, prm: GAParams, seed: int, gen: int) -> list:
    """Simple: the n_parents best.  Roulette: probability proportional to
    f - min(0, min f).  Tournament: k entrants without replacement from the
    ranking, the r-th best of them wins with probability q (1 - q)^r."""
    P = len(fit)
    parents = []
    if prm.selection == SEL_ROULETTE:
        vals = [0.0 if np.isnan(np.float32(f)) else float(np.float32(f)) for f in fit]
        lo = min(0.0, min(vals))
        cum, c = [], 0.0
        for v in vals:  # prefix sum in index order
            c += v - lo
            cum.append(c)
    for t in range(prm.n_parents):
        d = Draws(seed, t, gen, PURPOSE_SELECT)
        if prm.selection == SEL_SIMPLE:
            parents.append(order[t])
        elif prm.selection == SEL_ROULETTE:
            total = cum[-1]
            if not total > 0.0:
                parents.append(d.pick(P))
                continue
            target = (d.word() >> 8) * 2.0 ** -24 * total
            i = next((i for i in range(P) if cum[i] >= target), P - 1)
            parents.append(i)
        else:
            K = prm.tournament_k
            chosen = []
            for j in range(P - K, P):  # Floyd's sampling of K distinct positions
                r = d.pick(j + 1)
                chosen.append(j if r in chosen else r)
            chosen.sort()
            r = 0
            while r < K - 1 and d.u() >= f32(prm.tournament_q):
                r += 1
            parents.append(order[chosen[r]])
    return parents


# ----------------------------------------------------------------------------- guards
def free_slots(v, gap: int) -> list:
    occ = [s for s in range(len(v)) if v[s] > 0]
    return [s for s in range(len(v)) if all(abs(o - s) >= gap for o in occ)]


def repair(v, prm: GAParams, d: Draws):
    """Clip to d_max; relocate (or fold) doses closer than min_gap to the
    previous fraction; take one unit from the largest dose (earliest) until the
    total is within the cap."""
    for s in range(len(v)):
        v[s] = min(v[s], prm.d_max)
    while True:
        occ = [s for s in range(len(v)) if v[s] > 0]
        bad = [(a, j) for a, j in zip(occ[:-1], occ[1:]) if j - a < prm.min_gap]
        if not bad:
            break
        a, j = bad[0]
        dose = v[j]
        v[j] = 0
        free = free_slots(v, prm.min_gap)
        if free:
            v[free[d.pick(len(free))]] = dose
        else:
            v[a] = min(prm.d_max, v[a] + dose)
    while sum(v) > prm.total_cap:
        j = max(range(len(v)), key=lambda s: (v[s], -s))
        v[j] -= 1


# ----------------------------------------------------------------------------- mutation
def mutate(v, prm: GAParams, d: Draws):
    S = len(v)
    for bit in (MUT_SWAP, MUT_SPLIT, MUT_DOSE_TIME, MUT_DOSE_VALUE):
        if not prm.mutations & bit:
            continue
        if not d.u() < f32(prm.p_mut):
            continue
        occ = [s for s in range(S) if v[s] > 0]
        if bit == MUT_SWAP:
            if not occ:
                continue
            i = occ[d.pick(len(occ))]
            j = d.pick(S)
            v[i], v[j] = v[j], v[i]
        elif bit == MUT_SPLIT:
            big = [s for s in range(S) if v[s] > 1]
            if not big:
                continue
            i = big[d.pick(len(big))]
            part = 1 + d.pick(v[i] - 1)
            rest = v[i] - part
            v[i] = 0
            for dose in (part, rest):
                for _ in range(8):
                    j = d.pick(S)
                    if v[j] + dose <= prm.d_max:
                        v[j] += dose
                        break
                else:
                    v[i] += dose
        elif bit == MUT_DOSE_TIME:
            if not occ:
                continue
            i = occ[d.pick(len(occ))]
            j = d.pick(S)
            moved = max(0, min(v[i], prm.d_max - v[j])) if j != i else 0
            v[j] += moved
            v[i] -= moved
        else:
            slack = prm.total_cap - sum(v)
            if slack <= 0 or not occ:
                continue
            i = occ[d.pick(len(occ))]
            room = min(slack, prm.d_max - v[i])
            if room > 0:
                v[i] += 1 + d.pick(room)


# ----------------------------------------------------------------------------- crossover and children
def child_pair(pop, parents, m: int, prm: GAParams, seed: int, gen: int, rows: int):
    """The children of pair m (the first `rows` of the two are built)."""
    S = prm.n_slots
    d = Draws(seed, m, gen, PURPOSE_CHILD)
    npar = prm.n_parents
    ap = d.pick(npar)
    bq = d.pick(npar - 1 if npar > 1 else 1)
    bp = bq + (bq >= ap) if npar > 1 else ap
    A, B = [int(x) for x in pop[parents[ap]]], [int(x) for x in pop[parents[bp]]]
    if prm.crossover == X_UNIFORM:
        take_a = [d.u() < 0.5 for _ in range(S)]
    else:
        if prm.crossover == X_SINGLE:
            c1, c2 = S // 4 + d.pick(3 * S // 4 - S // 4 + 1), S
        else:
            c1 = S // 4 + d.pick(S // 2 - S // 4 + 1)
            c2 = S // 2 + d.pick(3 * S // 4 - S // 2 + 1)
        take_a = [s < c1 or s >= c2 for s in range(S)]
    c0 = [A[s] if take_a[s] else B[s] for s in range(S)]
    c1_ = [B[s] if take_a[s] else A[s] for s in range(S)]
    out = []
    for c in (c0, c1_)[:rows]:
        mutate(c, prm, d)
        repair(c, prm, d)
        out.append(np.array(c, dtype=np.uint8))
    return out


def generation(pop, fit, prm: GAParams, seed: int, gen: int, pairs=None):
    """Next population (elites, then children).  `pairs` limits the children
    built to those pair indices (rows not built stay zero)."""
    P, S = pop.shape
    order = ranking(fit)
    parents = select_parents(fit, order, prm, seed, gen)
    nxt = np.zeros_like(pop)
    for r in range(prm.n_elite):
        nxt[r] = pop[order[r]]
    n_children = P - prm.n_elite
    n_pairs = (n_children + 1) // 2
    for m in (range(n_pairs) if pairs is None else pairs):
        r0 = prm.n_elite + 2 * m
        rows = min(2, P - r0)
        for h, c in enumerate(child_pair(pop, parents, m, prm, seed, gen, rows)):
            nxt[r0 + h] = c
    return nxt, order, parents


def random_population(P: int, prm: GAParams, seed: int) -> np.ndarray:
    """Row i: 1 + pick(S / min_gap) fractions of 1 + pick(d_max) units at random slots, then the guards."""
    S = prm.n_slots
    pop = np.zeros((P, S), dtype=np.uint8)
    for i in range(P):
        d = Draws(seed, i, 0, PURPOSE_INIT)
        v = [0] * S
        for _ in range(1 + d.pick(S // prm.min_gap)):
            s = d.pick(S)
            v[s] = min(255, v[s] + 1 + d.pick(prm.d_max))
        repair(v, prm, d)
        pop[i] = v
    return pop


def is_valid(v, prm: GAParams) -> bool:
    occ = [s for s in range(len(v)) if v[s] > 0]
    gaps_ok = all(j - a >= prm.min_gap for a, j in zip(occ[:-1], occ[1:]))
    return gaps_ok and max(v, default=0) <= prm.d_max and sum(int(x) for x in v) <= prm.total_cap
