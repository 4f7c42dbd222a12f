"""Tumour case library and multi-tumour fitness (GPU)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_08123_b300 import _build
    _build.build()
    return torch


def test_library_growth_and_multi_tumour_fitness(cuda):
    from paper_2303_08123_b300 import Simulator, csr, library
    lib = library.grow_library(3, 24, 3, 12, seed=21)
    cells = [lib.get_state(t)[3] for t in range(3)]
    n0 = 123  # lattice points of a radius-3 ball
    live = [int(np.count_nonzero(c & 7)) for c in cells]
    assert all(x > n0 for x in live)  # untreated tumours grew
    assert not np.array_equal(cells[0], cells[1])  # each from its own seeded spheroid
    prot = [([4.0, 4.0], [0.5, 1.0]), ([], [])]
    mean, std, counts = library.evaluate(prot, lib, replicates=2, seed=5, regrowth_h=2)
    assert counts.shape == (2, 3, 2)
    assert mean[0] > mean[1]  # 8 Gy lowers the count, i.e. raises f = 1500 - n
    # a slot started by device copy equals one started from the same host arrays
    a = Simulator([24], [-1], seed=5, regrowth_h=2)
    b = Simulator([24], [-1], seed=5, regrowth_h=2)
    for s in (a, b):
        s.load_protocols(*csr([prot[0]]))
    a.copy_lattice(0, lib, 1)
    b.set_state(0, *lib.get_state(1))
    for s in (a, b):
        s.run(0)
    for x, y in zip(a.get_state(0), b.get_state(0)):
        assert np.array_equal(x, y)


def _oracle_continue(orc, p, state, seed, word, doses, waits, T, hours):
    """The oracle from a given state: T steps of or_step in order, fractions at
    their steps (600 x cumulative wait), live counts at every whole hour."""
    st = state.copy()
    fs = orc.fraction_steps(waits) if len(waits) else []
    counts = [-1] * (hours + 1)
    live = st.n_live()
    for s in range(T):
        if s % 600 == 0 and s // 600 <= hours:
            counts[s // 600] = live
        dose = sum(d for d, f in zip(doses, fs) if f == s)
        _, stats = orc.step(p, st, seed, word, s, dose=dose)
        live = stats["n_live"]
    if T % 600 == 0 and T // 600 <= hours:
        counts[T // 600] = live
    return st, np.array(counts)


def test_library_cases_equal_the_oracle(cuda, orc):
    """Library cases against the oracle: each case grown on the device equals
    the oracle's growth of the same seeded spheroid (cells bit for bit), and a
    protocol evaluated on the cases (device copies into its slots, two
    replicate slots per case) equals the oracle continued from the same
    grown state with the slot's protocol word: final cells and every hourly
    count."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2303_08123_b300 import library
    from synth.params import P0
    L, R, grow_h, seed_lib, seed_eval = 24, 3, 12, 21, 5
    lib = library.grow_library(2, L, R, grow_h, seed=seed_lib)
    for t in range(2):
        ref = orc.run(P0, L, R, seed_lib, t, [], [], t_end_steps=grow_h * 600, init_word=t)
        assert ref["stats"]["n_near"] == 0
        assert np.array_equal(lib.get_state(t)[3], ref["state"].cell), t
    prot = [([3.0, 2.0], [0.5, 1.0])]
    regrow = 2
    T = int(round(600 * 1.5)) + 600 * regrow
    hours = T // 600
    sim, slots = library.evaluation_batch(prot, lib, 2, seed_eval, regrowth_h=regrow, hours=hours)
    sim.run(0)
    grown = {}
    for t in range(2):
        O, G, H, cell = lib.get_state(t)
        st = orc.State(L)
        st.O[:], st.G[:], st.H[:], st.cell[:] = O, G, H, cell
        grown[t] = st
    with ThreadPoolExecutor(len(slots)) as ex:
        futs = [ex.submit(_oracle_continue, orc, P0, grown[t], seed_eval, k, prot[p][0], prot[p][1], T, hours)
                for k, (p, t, _) in enumerate(slots)]
        refs = [f.result() for f in futs]
    counts = sim.counts()
    for k, (st, cref) in enumerate(refs):
        O, G, H, cell = sim.get_state(k)
        assert np.array_equal(cell, st.cell), k
        assert np.array_equal(counts[k], cref), (k, counts[k], cref)
        for g, o, m in zip((O, G, H), (st.O, st.G, st.H), (P0.medium_O, P0.medium_G, 10 ** (3 - P0.medium_pH))):
            assert np.max(np.abs(g - o)) / m < 1e-4
    assert not np.array_equal(sim.get_state(0)[3], sim.get_state(1)[3])  # replicates differ


def test_paper_shaped_library(cuda):
    """The library in the paper's shape (ten tumours grown 240 h from radius-4
    seed balls on 48^3 lattices), evaluated with eight replicates per tumour in
    one batch: every tumour grew, the tumours differ, and a treated protocol
    scores better than no treatment over the 80 slots."""
    from paper_2303_08123_b300 import library
    lib = library.paper_library(seed=31)
    live = [int(np.count_nonzero(lib.get_state(t)[3] & 7)) for t in range(library.PAPER_CASES)]
    assert min(live) > 257 * 4, live
    assert len(set(live)) > 1
    prot = [([5.0, 5.0, 5.0], [0.0, 24.0, 24.0]), ([], [])]
    mean, std, counts = library.evaluate(prot, lib, library.PAPER_REPLICATES, seed=7, regrowth_h=6)
    assert counts.shape == (2, library.PAPER_CASES, library.PAPER_REPLICATES)
    assert mean[0] > mean[1] and np.all(std >= 0)
