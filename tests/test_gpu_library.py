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
