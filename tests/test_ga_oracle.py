"""Pins of the GA oracle (oracle/ga.py) to what the paper's GA operator
definitions fix ("The Genetic Algorithm (GA)", "The Main GA Loop", GA operator
details), on the CPU: validity under the guards, elitism, the selection laws
(a certain tournament, roulette shares, simple = sort), crossover conserving
the parents' genes slot by slot, mutations conserving the total dose, and hand
cases of the guards."""
import numpy as np
import pytest
from scipy import stats as sps

from oracle import ga as oga

SEED = 0x0DD5_EED5


def _distinct_population(P, prm, seed):
    pop = oga.random_population(P, prm, seed)
    assert len({bytes(r) for r in pop}) == P
    return pop


def test_random_population_is_valid_and_varied():
    prm = oga.GAParams(n_slots=240, d_max=8, total_cap=40, min_gap=12)
    pop = oga.random_population(48, prm, SEED)
    assert all(oga.is_valid(r, prm) for r in pop)
    assert all(r.sum() > 0 for r in pop)
    assert len({bytes(r) for r in pop}) == 48


def test_ranking_is_a_stable_descending_sort_with_nan_last():
    rng = np.random.default_rng(1)
    fit = rng.integers(-5, 5, size=200).astype(np.float32)
    fit[[3, 77]] = np.nan
    order = oga.ranking(fit)
    key = np.where(np.isnan(fit), -np.inf, fit)
    ref = np.lexsort((np.arange(200), -key))  # primary: fitness descending; ties: lower index
    assert order[:198] == [i for i in ref if not np.isnan(fit[i])]
    assert order[198:] == [3, 77]


def test_elites_are_the_best_and_every_child_is_valid():
    prm = oga.GAParams(n_slots=96, d_max=8, total_cap=24, min_gap=6, n_elite=3, n_parents=8,
                       mutations=oga.MUT_SWAP | oga.MUT_SPLIT | oga.MUT_DOSE_TIME | oga.MUT_DOSE_VALUE, p_mut=0.7)
    pop = _distinct_population(33, prm, SEED)
    fit = np.random.default_rng(2).normal(size=33).astype(np.float32)
    nxt, order, parents = oga.generation(pop, fit, prm, SEED, 1)
    best = np.argsort(-fit, kind="stable")
    for r in range(3):
        assert np.array_equal(nxt[r], pop[best[r]])
    assert parents == list(best[:8])  # simple selection: the n_parents best
    assert all(oga.is_valid(r, prm) for r in nxt)


def test_certain_tournaments_pick_the_best_or_the_worst():
    """k = P entrants: with q = 1 the best always wins, with q = 0 the walk
    runs to the last entrant, i.e. the worst individual."""
    prm = oga.GAParams(n_slots=48, min_gap=4, n_parents=20, selection=oga.SEL_TOURNAMENT, tournament_k=20)
    fit = np.random.default_rng(3).normal(size=20).astype(np.float32)
    order = oga.ranking(fit)
    prm.tournament_q = 1.0
    assert oga.select_parents(fit, order, prm, SEED, 0) == [order[0]] * 20
    prm.tournament_q = 0.0
    assert oga.select_parents(fit, order, prm, SEED, 0) == [order[-1]] * 20


def test_tournament_winner_rank_follows_the_geometric_law():
    """k = 4 of P = 4 entrants (the whole population), q = 0.5: the r-th best
    wins with probability q (1 - q)^r, the last takes the rest."""
    prm = oga.GAParams(n_slots=48, min_gap=4, n_parents=4, selection=oga.SEL_TOURNAMENT, tournament_k=4,
                       tournament_q=0.5)
    fit = np.array([3.0, 1.0, 4.0, 2.0], dtype=np.float32)
    order = oga.ranking(fit)
    counts = np.zeros(4)
    for g in range(1500):
        for w in oga.select_parents(fit, order, prm, SEED, g):
            counts[order.index(w)] += 1
    q = 0.5
    p = np.array([q, q * (1 - q), q * (1 - q) ** 2, (1 - q) ** 3])
    assert sps.chisquare(counts, p * counts.sum()).pvalue > 1e-4


def test_roulette_shares_follow_the_shifted_fitness():
    P = 2000
    prm = oga.GAParams(n_slots=48, min_gap=4, n_parents=P, selection=oga.SEL_ROULETTE)
    fit = np.zeros(P, dtype=np.float32)
    fit[:4] = [1, 2, 3, 4]
    sel = oga.select_parents(fit, oga.ranking(fit), prm, SEED, 0)
    counts = np.bincount(sel, minlength=P)
    assert counts[4:].sum() == 0
    assert sps.chisquare(counts[:4], np.array([.1, .2, .3, .4]) * P).pvalue > 1e-4
    # negative fitness: shifted by the minimum, so the least fit gets nothing
    fit2 = np.full(P, -1.0, dtype=np.float32)
    fit2[:2] = [0.0, 1.0]
    sel2 = oga.select_parents(fit2, oga.ranking(fit2), prm, SEED, 1)
    c2 = np.bincount(sel2, minlength=P)
    assert c2[2:].sum() == 0 and sps.chisquare(c2[:2], [P / 3, 2 * P / 3]).pvalue > 1e-4


@pytest.mark.parametrize("cross", [oga.X_SINGLE, oga.X_TWO, oga.X_UNIFORM])
def test_crossover_conserves_genes_and_respects_cut_ranges(cross):
    """No mutation and guards that cannot bind (min_gap 1, cap above any sum):
    each child slot comes from one parent and the pair together holds exactly
    the parents' genes; single and two-point cuts lie in the stated ranges."""
    S = 64
    prm = oga.GAParams(n_slots=S, d_max=8, total_cap=10_000, min_gap=1, n_elite=0, n_parents=6, crossover=cross,
                       mutations=0)
    rng = np.random.default_rng(4)
    pop = rng.integers(0, 9, size=(12, S)).astype(np.uint8)
    fit = rng.normal(size=12).astype(np.float32)
    nxt, order, parents = oga.generation(pop, fit, prm, SEED, 5)
    for m in range(6):
        c0, c1 = nxt[2 * m].astype(int), nxt[2 * m + 1].astype(int)
        pairs = [(a, b) for a in parents for b in parents
                 if np.array_equal(c0 + c1, pop[a].astype(int) + pop[b].astype(int))
                 and np.all((c0 == pop[a]) | (c0 == pop[b]))]
        assert pairs, m
        ok = False
        for a, b in pairs:
            A, B = pop[a], pop[b]
            if cross == oga.X_UNIFORM:
                ok |= bool(np.all(((c0 == A) & (c1 == B)) | ((c0 == B) & (c1 == A))))
                continue
            cut_sets = ([(c, S) for c in range(S // 4, 3 * S // 4 + 1)] if cross == oga.X_SINGLE else
                        [(x, y) for x in range(S // 4, S // 2 + 1) for y in range(S // 2, 3 * S // 4 + 1)])
            for x, y in cut_sets:
                inside = (np.arange(S) >= x) & (np.arange(S) < y)
                if np.array_equal(c0, np.where(inside, B, A)) and np.array_equal(c1, np.where(inside, A, B)):
                    ok = True
                    break
        assert ok, m


@pytest.mark.parametrize("mut", [oga.MUT_SWAP, oga.MUT_SPLIT, oga.MUT_DOSE_TIME, oga.MUT_DOSE_VALUE])
def test_mutations_conserve_or_bound_the_total_dose(mut):
    """swap, split and dose-time move dose around without changing the pair's
    total; dose-value only adds dose, and never beyond the cap."""
    S = 64
    cap = 10_000 if mut != oga.MUT_DOSE_VALUE else 60
    prm = oga.GAParams(n_slots=S, d_max=8, total_cap=cap, min_gap=1, n_elite=0, n_parents=4,
                       crossover=oga.X_SINGLE, mutations=mut, p_mut=1.0)
    rng = np.random.default_rng(5)
    pop = (rng.integers(0, 9, size=(8, S)) * (rng.random((8, S)) < 0.15)).astype(np.uint8)
    fit = rng.normal(size=8).astype(np.float32)
    nxt, _, parents = oga.generation(pop, fit, prm, SEED, 2)
    changed = 0
    for m in range(4):
        c0, c1 = nxt[2 * m].astype(int), nxt[2 * m + 1].astype(int)
        tot = c0.sum() + c1.sum()
        parent_tots = {int(pop[a].sum()) + int(pop[b].sum()) for a in parents for b in parents if a != b}
        if mut == oga.MUT_DOSE_VALUE:
            assert c0.sum() <= cap and c1.sum() <= cap
            changed += tot not in parent_tots
        else:
            assert tot in parent_tots
        assert c0.max() <= 8 and c1.max() <= 8
    if mut == oga.MUT_DOSE_VALUE:
        assert changed > 0


def test_guards_on_hand_cases():
    d = oga.Draws(SEED, 0, 0, oga.PURPOSE_CHILD)
    # total cap: one unit at a time from the largest dose, earliest first
    v = [4, 4, 2]
    oga.repair(v, oga.GAParams(n_slots=3, d_max=8, total_cap=7, min_gap=1), d)
    assert v == [2, 3, 2]
    # interval: the only free slot keeps every gap
    v = [2, 0, 1, 0]
    oga.repair(v, oga.GAParams(n_slots=4, d_max=8, total_cap=99, min_gap=3), d)
    assert v == [2, 0, 0, 1]
    # no free slot: folded into the previous fraction, capped at d_max
    v = [2, 0, 1]
    oga.repair(v, oga.GAParams(n_slots=3, d_max=8, total_cap=99, min_gap=3), d)
    assert v == [3, 0, 0]
    v = [2, 0, 1]
    oga.repair(v, oga.GAParams(n_slots=3, d_max=2, total_cap=99, min_gap=3), d)
    assert v == [2, 0, 0]
    # clip first
    v = [9, 0, 0, 0]
    oga.repair(v, oga.GAParams(n_slots=4, d_max=8, total_cap=99, min_gap=1), d)
    assert v == [8, 0, 0, 0]


@pytest.mark.parametrize("cross", [oga.X_SINGLE, oga.X_TWO])
def test_crossover_cut_points_cover_exactly_the_stated_ranges(cross):
    """Two parents that differ in every slot make each child pair's cut points
    readable: every cut lies in its stated range and, over 300 pairs, both ends
    of each range occur (single point: [S/4, 3S/4]; two points: [S/4, S/2] and
    [S/2, 3S/4])."""
    S = 64
    prm = oga.GAParams(n_slots=S, d_max=8, total_cap=10_000, min_gap=1, n_elite=0, n_parents=2, crossover=cross,
                       mutations=0)
    P = 600
    pop = np.zeros((P, S), dtype=np.uint8)
    pop[:, :] = 1
    pop[0] = 1 + np.arange(S) % 4
    pop[1] = 5 + np.arange(S) % 4
    fit = np.zeros(P, dtype=np.float32)
    fit[:2] = [2.0, 1.0]  # the two parents
    nxt, _, parents = oga.generation(pop, fit, prm, SEED, 4)
    assert sorted(parents) == [0, 1]
    c1s, c2s = [], []
    for m in range(P // 2):
        c0 = nxt[2 * m]
        a_first = c0[0] == pop[0][0]
        other = pop[1] if a_first else pop[0]
        inside = np.flatnonzero(c0 == other)
        if cross == oga.X_SINGLE:
            assert inside.size and inside[-1] == S - 1 and np.array_equal(inside, np.arange(inside[0], S))
            c1s.append(int(inside[0]))
        else:
            if inside.size == 0:  # c1 == c2: no middle segment
                continue
            assert np.array_equal(inside, np.arange(inside[0], inside[-1] + 1))
            c1s.append(int(inside[0]))
            c2s.append(int(inside[-1]) + 1)
    if cross == oga.X_SINGLE:
        assert min(c1s) == S // 4 and max(c1s) == 3 * S // 4
    else:
        assert min(c1s) == S // 4 and max(c1s) == S // 2
        assert min(c2s) == S // 2 and max(c2s) == 3 * S // 4
