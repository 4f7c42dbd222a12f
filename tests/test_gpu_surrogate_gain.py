"""What the trained surrogate gains (GPU).

The surrogate is trained on 2,048 simulated protocols.  From a fresh pool of
4,096 candidates it promotes the 256 it predicts best; the same number of
candidates drawn at random is the method without it.  Both sets are scored by
the full simulator: the promoted set must contain clearly better protocols
(lower final live counts, a t-test far beyond chance), so the same search
quality needs far fewer full simulations.  Its predictions must also rank a
held-out set in the simulator's order (Spearman correlation).
"""
import numpy as np
import pytest
from scipy import stats as sps

from synth import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_08123_b300 import _build
    _build.build()
    return torch


def _protocols(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        k = int(rng.integers(2, 7))
        d = rng.choice([0.5, 1.0, 1.5, 2.0, 2.5], size=k).tolist()
        w = rng.choice([0.5, 1.0, 2.0, 3.0, 4.0], size=k).tolist()
        out.append((workloads.cap_total_dose(d, 8.0, 0.5), w))
    return out


def test_surrogate_promotes_better_protocols_than_random(cuda):
    from paper_2303_08123_b300.screen import SimSetup, features, fit_surrogate, simulate
    from paper_2303_08123_b300.surrogate import Surrogate
    setup = SimSetup(L=24, R=5, regrowth_h=6)
    train = _protocols(2048, 1)
    y = simulate(train, setup)
    net = Surrogate(batch_max=4096, seed=3)
    mu, sd = fit_surrogate(net, features(train), y, epochs=60)
    held = _protocols(512, 2)
    y_held = simulate(held, setup, seed_offset=100)
    rho = sps.spearmanr(net.predict(features(held)), y_held).correlation
    assert rho > 0.6, rho
    pool = _protocols(4096, 3)
    pred = net.predict(features(pool))
    promoted = [pool[i] for i in np.argsort(pred, kind="stable")[:256]]
    rng = np.random.default_rng(4)
    random_pick = [pool[i] for i in rng.choice(len(pool), 256, replace=False)]
    yp = simulate(promoted, setup, seed_offset=200)
    yr = simulate(random_pick, setup, seed_offset=300)
    t = sps.ttest_ind(yp, yr, alternative="less")
    assert yp.mean() < yr.mean() and t.pvalue < 1e-6, (yp.mean(), yr.mean(), t.pvalue)
    # the promoted set's best equals what random sampling needs many more simulations to reach
    assert yp.min() <= np.sort(yr)[2]


def test_screened_ga_reaches_the_plain_best_with_fewer_simulations(cuda):
    """Equal best fitness with fewer full simulations, training included: the
    plain GA simulates 256 children per generation for 10 generations; the
    screened GA ranks 2,048 candidates per generation with a surrogate trained
    on 1,024 simulated random protocols and simulates the best 128.  The
    screened arm's simulations until its best-so-far count first reaches the
    plain GA's final best (its 1,024 training simulations counted) must be
    fewer than the plain GA's own."""
    from paper_2303_08123_b300 import ga
    from paper_2303_08123_b300.screen import SimSetup, compare_arms
    setup = SimSetup(L=24, R=5, regrowth_h=6)
    cfg = ga.GAConfig(n_slots=48, d_max=2.5, total_cap=8.0, min_gap=4,
                      mutations=("swap", "split", "dose_time", "dose_value"), p_mut=0.5)
    r = compare_arms(setup, cfg, generations=10, plain_population=256, simulated=128, pool=2048, train=1024, seed=5)
    assert r["screened_sims_to_best"] is not None, r
    assert r["screened_sims_to_best"] < r["plain_sims_to_best"], (r["target"], r["plain_sims_to_best"],
                                                                  r["screened_sims_to_best"])
