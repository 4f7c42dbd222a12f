"""Host GA (CPU): encoding, guards, selection laws, crossover ranges and the
constraints every operator must keep."""
import json
import os

import numpy as np
import pytest

from paper_2303_08123_b300 import ga


def test_sparse_vector_round_trip_matches_paper_examples():
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "benchmark_protocols.json")))
    for entry in gold["protocols"].values():
        doses = [d for d, _ in entry["pairs"]]
        waits = [w for _, w in entry["pairs"]]
        vec = ga.from_pairs(doses, waits, gold["sparse_example"]["length"])
        assert list(np.flatnonzero(vec)) == entry["slots_30min"]
        d2, w2 = ga.to_pairs(vec)
        assert d2 == doses and w2 == waits
    ex = gold["sparse_example"]
    vec = np.zeros(ex["length"])
    vec[ex["position"]] = ex["dose_gy"]
    d, w = ga.to_pairs(vec)
    assert d == [ex["dose_gy"]] and w == [ex["hours_after_start"]]


def test_total_guard_removes_quarter_gray_from_largest():
    cfg = ga.GAConfig(total_cap=10.0, d_max=5.0)
    vec = np.zeros(240)
    vec[[0, 20, 40]] = [5.0, 4.0, 3.0]  # 12 Gy
    out = ga.guard_total(vec, cfg)
    assert out.sum() == 10.0
    # 8 decrements, always from the current maximum, earliest on ties
    assert list(out[[0, 20, 40]]) == [3.5, 3.5, 3.0]


def test_interval_guard_restores_minimum_gap():
    cfg = ga.GAConfig(min_gap=12)
    rng = np.random.default_rng(0)
    vec = np.zeros(240)
    vec[[10, 12, 14, 100]] = 1.0
    out = ga.guard_interval(vec, cfg, rng)
    idx = np.flatnonzero(out)
    assert np.all(np.diff(idx) >= 12) and abs(out.sum() - 4.0) < 1e-12
    crowded = np.zeros(24)
    crowded[[0, 1, 2]] = 0.5  # no room for three fractions 12 slots apart in 24 slots
    out = ga.guard_interval(crowded, ga.GAConfig(n_slots=24, min_gap=12, d_max=2.0), rng)
    assert np.all(np.diff(np.flatnonzero(out)) >= 12)


@pytest.mark.parametrize("sel", ["simple", "roulette", "tournament"])
@pytest.mark.parametrize("cx", ["single_point", "two_point", "uniform"])
def test_generations_keep_every_constraint(sel, cx):
    cfg = ga.GAConfig(selection=sel, crossover=cx, mutations=("swap", "split", "dose_time", "dose_value"),
                      p_mut=0.8, d_max=2.5)
    rng = np.random.default_rng(1)
    pop = [ga.random_protocol(cfg, rng) for _ in range(40)]
    for _ in range(5):
        fit = rng.random(40)
        elites, children = ga.next_generation(pop, fit, cfg, rng)
        assert len(elites) == 4 and len(children) == 36
        pop = elites + children
        for p in pop:
            assert ga.is_valid(p, cfg)


def test_simple_selection_and_elitism_take_the_best():
    fit = np.array([3.0, 9.0, 1.0, 7.0, 5.0])
    assert ga.select_simple(fit, 2) == [1, 3]
    cfg = ga.GAConfig(population=5, elite_frac=0.2)
    rng = np.random.default_rng(0)
    pop = [np.full(240, i, dtype=float) for i in range(5)]
    elites, _ = ga.next_generation([ga.random_protocol(cfg, rng) for _ in range(5)], fit, cfg, rng)
    assert len(elites) == 1


def test_roulette_is_fitness_proportional():
    rng = np.random.default_rng(2)
    fit = np.array([1.0, 2.0, 3.0, 4.0])
    picks = np.bincount(ga.select_roulette(fit, 40000, rng), minlength=4) / 40000
    np.testing.assert_allclose(picks, fit / fit.sum(), atol=0.01)


def test_tournament_prefers_better_ranks_with_geometric_law():
    rng = np.random.default_rng(3)
    fit = np.arange(16, dtype=float)  # index 15 is the best
    picks = np.bincount(ga.select_tournament(fit, 20000, rng, k=16, q=0.9), minlength=16) / 20000
    # with all 16 entering, rank r wins with probability q (1 - q)^r (the last rank takes the rest)
    want = [0.9 * 0.1 ** r for r in range(15)]
    want.append(1 - sum(want))
    np.testing.assert_allclose(picks[::-1], want, atol=0.01)


def test_crossover_points_stay_in_the_paper_ranges():
    rng = np.random.default_rng(4)
    a, b = np.zeros(240), np.ones(240)
    for _ in range(200):
        c, _ = ga.crossover(a, b, "single_point", rng)
        cut = int(np.argmax(c > 0))
        assert 60 <= cut <= 180
        c, d = ga.crossover(a, b, "two_point", rng)
        mid = np.flatnonzero(c > 0)
        assert 60 <= mid[0] <= 120 and 120 <= mid[-1] + 1 <= 180
        assert np.array_equal(c + d, np.ones(240))
        u, v = ga.crossover(a, b, "uniform", rng)
        assert np.array_equal(u + v, np.ones(240))
