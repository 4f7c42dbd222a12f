"""Statistical parity, precision variants and device-side mass sums (GPU).

* 64 replicate simulations of one protocol on the GPU and 64 on the FP64 oracle
  with a different Philox key (independent samples of the same stochastic
  model, each replicate with its own seeded spheroid): the mean final count
  agrees within 1 % and a two-sample Kolmogorov-Smirnov test does not reject.
* BF16 / FP16 field storage (FP32 arithmetic) against the FP64 oracle: field
  error and final-count error stay within stated bounds.
* Per-protocol substrate totals: FP64 on the device equals an FP64 host sum of
  the same values; the Kahan FP32 sum is within a few FP32 ulps of it.
"""
import numpy as np
import pytest
from scipy import stats as sps

from synth.params import P0
from synth import workloads
from tests import _parity as par

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_08123_b300 import _build
    _build.build()
    return torch


def test_replicates_match_oracle_distribution(cuda, orc):
    from paper_2303_08123_b300 import Simulator, csr
    n, L, R, T = 64, 24, 5, 7200  # 12 h, fractions at 1 h and 6 h
    doses, waits = [2.0, 2.0], [1.0, 5.0]
    sim = Simulator([L] * n, [R] * n, seed=0xA11CE, init_word=0xFFFFFFFE, t_end_steps=T)
    sim.load_protocols(*csr([(doses, waits)] * n))
    sim.run(0)
    g, _ = sim.fitness()
    off, d, w = csr([(doses, waits)] * n)
    ref = orc.run_batch(P0, [L] * n, [R] * n, 0xB0B, off, d, w, t_end_steps=T, init_word=0xFFFFFFFE)
    o = ref["n_final"]
    assert np.std(g) > 0 and np.std(o) > 0
    rel = abs(g.mean() - o.mean()) / o.mean()
    ks = sps.ks_2samp(g, o)
    assert rel < 0.01, (g.mean(), o.mean(), g.std(), o.std())
    assert ks.pvalue > 0.01, ks


def test_whole_trajectories_match_oracle_distribution(cuda):
    """Whole trajectories over the paper's horizon: 64 GPU replicates of the
    benchmark protocol BMII (5 x 2 Gy daily from t = 0) for ten days (240 h,
    144,000 steps) on 24^3 lattices, each growing its own seeded spheroid,
    against the final counts of 64 oracle replicates drawn under another key
    (tests/golden/replicates_240h.json, written from oracle/ alone by
    make_replicates_golden.py): mean final count within 1 %, two-sample KS
    p > 0.01."""
    import json
    import os
    from paper_2303_08123_b300 import Simulator, csr
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "replicates_240h.json")) as f:
        ref = json.load(f)
    doses, waits = workloads.benchmark_bmii()
    assert ref["doses"] == doses and ref["waits"] == waits
    n, L, R, T = ref["n"], ref["L"], ref["R"], ref["hours"] * 600
    sim = Simulator([L] * n, [R] * n, seed=0xA11CE, init_word=0xFFFFFFFE, t_end_steps=T)
    sim.load_protocols(*csr([(doses, waits)] * n))
    sim.autotune(3)
    sim.run(0)
    g, _ = sim.fitness()
    o = np.array(ref["n_final"], dtype=np.float64)
    assert np.std(g) > 0 and np.std(o) > 0
    rel = abs(g.mean() - o.mean()) / o.mean()
    ks = sps.ks_2samp(g, o)
    print(f"whole trajectories: GPU mean {g.mean():.1f} sd {g.std():.1f}, oracle mean {o.mean():.1f} "
          f"sd {o.std():.1f}, relative difference {rel:.4f}, KS p {ks.pvalue:.3f}")
    assert rel < 0.01, (g.mean(), o.mean(), g.std(), o.std())
    assert ks.pvalue > 0.01, ks


@pytest.mark.parametrize("precision,field_tol,count_tol", [("bf16", 2.5e-2, 0.02), ("fp16", 5e-3, 0.01)])
def test_reduced_precision_storage_against_oracle(cuda, orc, precision, field_tol, count_tol):
    from paper_2303_08123_b300 import Simulator, csr
    n, L, R, T = 8, 32, 6, 1800
    prot = [([1.0 + 0.5 * (i % 3), 1.5], [0.5, 1.0]) for i in range(n)]
    sim = Simulator([L] * n, [R] * n, seed=77, precision=precision, t_end_steps=T, dose_cap_gy=20.0)
    sim.load_protocols(*csr(prot))
    sim.run(0)
    cnt, _ = sim.fitness()
    worst_f, worst_c = 0.0, 0.0
    for p in range(0, n, 2):
        ref = orc.run(P0, L, R, 77, p, prot[p][0], prot[p][1], t_end_steps=T)
        O, G, H, _ = sim.get_state(p)
        st = ref["state"]
        ferr = max(float(np.max(np.abs(a - b))) / m for a, b, m in zip((O, G, H), (st.O, st.G, st.H), par.medium()))
        cerr = abs(int(cnt[p]) - ref["stats"]["n_live"]) / ref["stats"]["n_live"]
        worst_f, worst_c = max(worst_f, ferr), max(worst_c, cerr)
    assert worst_f < field_tol, worst_f
    assert worst_c < count_tol, worst_c


def test_field_totals_fp64_and_kahan(cuda):
    from paper_2303_08123_b300 import Simulator
    L = [40, 24]
    sim = Simulator(L, [-1, -1])
    want = []
    for p, l in enumerate(L):
        fields, cell = par.random_state(l, 50 + p)
        fields = [f * np.float32(1.0 + 3.0 * (k == 1)) for k, f in enumerate(fields)]
        sim.set_state(p, *fields, cell)
        want.append([np.sum(f.astype(np.float64)) for f in fields])
    t64, t32 = sim.field_totals()
    want = np.array(want)
    np.testing.assert_allclose(t64, want, rtol=1e-13)
    np.testing.assert_allclose(t32.astype(np.float64), want, rtol=4e-7)
