"""The index-checking debug build (libsim_check.so, compiled with SIM_CHECK):
on the batches of the parity tests every kernel stays inside the batch (no
status bit is raised) and the results equal the normal build bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x0C4E_C4ED


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_08123_b300 import _build
    _build.build()
    return torch


@pytest.mark.parametrize("path,shape", [("fused", 3), ("fused", 4), ("fused", 1), ("fused", 5), ("fused", 6),
                                        ("fused", 7), ("fused", 8), ("substep", 0)])
def test_checked_build_stays_in_bounds_and_matches(cuda, path, shape):
    from paper_2303_08123_b300 import Simulator, csr
    from synth import workloads
    L, R, prot = workloads.ragged_batch(24, seed=21, r_min=3, r_max=10, f_min=2, f_max=6)
    prot = [(d, [0.5] + w[1:]) for d, w in prot]
    out = []
    for check in (False, True):
        sim = Simulator(L, R, seed=SEED, hours=2, t_end_steps=1500, path=path, tile_shape=shape, check=check)
        sim.load_protocols(*csr(prot))
        sim.run(0)
        n, _ = sim.fitness()  # raises if a checked kernel flagged an index
        out.append(([sim.get_state(p)[3] for p in range(len(L))], sim.counts(), n))
        sim.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_checked_build_bf16_pair_kernel(cuda):
    from paper_2303_08123_b300 import Simulator, csr
    from synth import workloads
    prot = workloads.ga_batch(8, seed=5)
    prot = [(d, [0.5] + w[1:]) for d, w in prot]
    sims = [Simulator([32] * 8, [6] * 8, seed=SEED, precision="bf16", t_end_steps=900, hours=1, check=c)
            for c in (False, True)]
    for sim in sims:
        sim.load_protocols(*csr(prot))
        sim.run(0)
        sim.fitness()
    for p in range(8):
        assert np.array_equal(sims[0].get_state(p)[3], sims[1].get_state(p)[3])
