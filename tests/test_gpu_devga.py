"""Device-resident GA (libga) and the device-side protocol loader against the
CPU oracle, through the C ABI.  Everything here is integer work, so the bar is
bit-exact: populations, rankings, fraction tables (via whole runs)."""
import numpy as np
import pytest

from oracle import ga as oga

pytestmark = pytest.mark.gpu

SEED = 0x5EED_0000_0000_6A6A


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_08123_b300 import _build
    _build.build()
    return torch


def _dev_params(p: oga.GAParams):
    from paper_2303_08123_b300.devga import make_params
    return make_params(**{k: getattr(p, k) for k in (
        "n_slots", "d_max", "total_cap", "min_gap", "n_elite", "n_parents", "selection", "crossover",
        "mutations", "p_mut", "tournament_k", "tournament_q")})


def _fitness(P, seed):
    rng = np.random.default_rng(seed)
    f = rng.integers(0, 40, size=P).astype(np.float32)  # ties on purpose
    f[P // 3] = np.nan
    f[P // 2] = -3.5
    return f


ALL_MUT = oga.MUT_SWAP | oga.MUT_SPLIT | oga.MUT_DOSE_TIME | oga.MUT_DOSE_VALUE


def test_random_population_bit_exact(cuda):
    from paper_2303_08123_b300.devga import DeviceGA
    prm = oga.GAParams(n_slots=240, d_max=8, total_cap=40, min_gap=12)
    dga = DeviceGA(_dev_params(prm), 97)
    got = dga.random_population(SEED).cpu().numpy()
    assert np.array_equal(got, oga.random_population(97, prm, SEED))


@pytest.mark.parametrize("sel,cross,mut,P,elite", [
    (oga.SEL_SIMPLE, oga.X_TWO, oga.MUT_SWAP | oga.MUT_SPLIT | oga.MUT_DOSE_TIME, 64, 6),
    (oga.SEL_ROULETTE, oga.X_SINGLE, ALL_MUT, 65, 3),
    (oga.SEL_TOURNAMENT, oga.X_UNIFORM, ALL_MUT, 50, 0),
    (oga.SEL_TOURNAMENT, oga.X_TWO, oga.MUT_DOSE_VALUE, 33, 33),
])
def test_generation_bit_exact(cuda, sel, cross, mut, P, elite):
    torch = cuda
    from paper_2303_08123_b300.devga import DeviceGA
    prm = oga.GAParams(n_slots=240, d_max=8, total_cap=40, min_gap=12, n_elite=elite, n_parents=max(2, P // 3),
                       selection=sel, crossover=cross, mutations=mut, p_mut=0.6, tournament_k=min(16, P),
                       tournament_q=0.75)
    pop = oga.random_population(P, prm, SEED ^ 1)
    fit = _fitness(P, 7)
    dga = DeviceGA(_dev_params(prm), P)
    nxt, order = dga.generation(torch.from_numpy(pop).cuda(), torch.from_numpy(fit).cuda(), SEED, 9)
    ref, ref_order, _ = oga.generation(pop, fit, prm, SEED, 9)
    assert order.cpu().tolist() == ref_order
    assert np.array_equal(nxt.cpu().numpy(), ref)
    assert all(oga.is_valid(r, prm) for r in ref)


@pytest.mark.parametrize("sel", [oga.SEL_SIMPLE, oga.SEL_ROULETTE, oga.SEL_TOURNAMENT])
def test_full_size_generation_sampled(cuda, sel):
    """Population 4,096 x 240 slots (the paper's 5-day vector at 30 min): the
    whole ranking, every elite, and sampled child pairs equal the oracle."""
    torch = cuda
    from paper_2303_08123_b300.devga import DeviceGA
    P = 4096
    prm = oga.GAParams(n_slots=240, d_max=8, total_cap=40, min_gap=12, n_elite=410, n_parents=1638,
                       selection=sel, crossover=oga.X_TWO, mutations=ALL_MUT, p_mut=0.3, tournament_k=16,
                       tournament_q=0.9)
    dga = DeviceGA(_dev_params(prm), P)
    pop_d = dga.random_population(SEED)
    pop = pop_d.cpu().numpy()
    fit = _fitness(P, 11)
    nxt, order = dga.generation(pop_d, torch.from_numpy(fit).cuda(), SEED, 3)
    nxt = nxt.cpu().numpy()
    n_pairs = (P - 410 + 1) // 2
    sample = [0, 1, 500, n_pairs - 1]
    ref, ref_order, _ = oga.generation(pop, fit, prm, SEED, 3, pairs=sample)
    assert order.cpu().tolist() == ref_order
    assert np.array_equal(nxt[:410], ref[:410])
    for m in sample:
        rows = [r for r in (410 + 2 * m, 411 + 2 * m) if r < P]
        assert np.array_equal(nxt[rows], ref[rows]), m
    assert all(oga.is_valid(r, prm) for r in nxt[::97])


def _sim(n, L=16, R=3, t_end=1200, **kw):
    from paper_2303_08123_b300 import Simulator
    return Simulator([L] * n, [R] * n, seed=SEED, t_end_steps=t_end, hours=2, dose_cap_gy=12.0, max_fractions=8,
                     **kw)


def _pairs(vec, unit_gy=0.25):
    from paper_2303_08123_b300 import ga
    return ga.to_pairs(np.asarray(vec, dtype=float) * unit_gy)


@pytest.mark.parametrize("half_h", [0.0, 1.0])
def test_device_loader_equals_host_loader(cuda, half_h):
    """Dose vectors loaded on the device run exactly like the same protocols
    given as host (dose, wait) lists."""
    torch = cuda
    from paper_2303_08123_b300 import csr
    from synth.params import P0
    prm = oga.GAParams(n_slots=8, d_max=16, total_cap=48, min_gap=2)
    pop = oga.random_population(24, prm, SEED)
    p = P0.replace(repair_half_h=half_h)
    a, b = _sim(24, params=p), _sim(24, params=p)
    a.load_dose_vectors(torch.from_numpy(pop).cuda())
    b.load_protocols(*csr([_pairs(r) for r in pop]))
    a.run(0)
    b.run(0)
    for i in range(24):
        assert np.array_equal(a.get_state(i)[3], b.get_state(i)[3]), i
    assert np.array_equal(a.counts(), b.counts())
    np.testing.assert_array_equal(a.delivered_dose(), b.delivered_dose())
    cnt, fit = a.fitness_device()
    n_host, f_host = b.fitness()
    assert np.array_equal(cnt.cpu().numpy(), n_host)
    assert np.array_equal(fit.cpu().numpy(), f_host.astype(np.float32))


def test_device_loader_rejects_rows_over_the_limits(cuda):
    torch = cuda
    from paper_2303_08123_b300 import SimError
    sim = _sim(2)
    rows = np.zeros((2, 8), dtype=np.uint8)
    rows[0, ::2] = 4            # 4 fractions x 1 Gy: fine
    rows[1, :] = 8              # 8 x 2 Gy = 16 Gy: above the 12 Gy cap
    sim.load_dose_vectors(torch.from_numpy(rows).cuda())
    sim.run(0)
    with pytest.raises(SimError):
        sim.fitness()
    rows[1, :] = 1
    sim.load_dose_vectors(torch.from_numpy(rows).cuda())  # a clean reload clears the error
    sim.run(0)
    sim.fitness()
    with pytest.raises(SimError):
        _sim(2, t_end=0).load_dose_vectors(torch.from_numpy(rows).cuda())  # needs a fixed horizon


def test_evolve_on_device_equals_host_orchestrated_loop(cuda):
    """Two generations with every step on the device equal the same loop
    driven from the host (oracle GA, host protocol lists, host fitness)."""
    torch = cuda
    from paper_2303_08123_b300 import csr
    from paper_2303_08123_b300.devga import DeviceGA, evolve_on_device
    P = 24
    prm = oga.GAParams(n_slots=8, d_max=8, total_cap=24, min_gap=2, n_elite=2, n_parents=8,
                       selection=oga.SEL_TOURNAMENT, crossover=oga.X_TWO, mutations=ALL_MUT, p_mut=0.5,
                       tournament_k=6, tournament_q=0.8)
    dga = DeviceGA(_dev_params(prm), P)
    sim = _sim(P)
    final, hist = evolve_on_device(sim, dga, 2, SEED)
    host = _sim(P)
    pop = oga.random_population(P, prm, SEED)
    for g in range(3):
        host.load_protocols(*csr([_pairs(r) for r in pop]))
        host.run(0)
        _, f = host.fitness()
        f = f.astype(np.float32)
        assert np.array_equal(hist[g].cpu().numpy(), f), g
        if g < 2:
            pop = oga.generation(pop, f, prm, SEED, g + 1)[0]
    assert np.array_equal(final.cpu().numpy(), pop)
