"""The allocation-free entry point sim_diffuse_noalloc against the context path.

Some callers cannot allocate device memory: hosts whose pool allocator owns all
of it, or latency-bound loops that cannot pay for cudaMalloc's synchronisation.
sim_diffuse_noalloc serves them with a fixed in-library scratch array.  Here it
must reproduce, call after call, the fields that sim_run computes for protocol
slot 0 on the same lattice, within the per-step field tolerance the other
parity tests use (the kernels are the same, so in practice bit for bit), and
apply the same irradiation marks to the cell words.

This file is named so that pytest collects it last: if it fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from synth.params import P0, F_REACTION, F_DIFFUSION
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


# (lattice side, substeps per step): the default case; an odd substep count,
# whose result the entry point copies back from its scratch array; and the
# largest lattice, which fills the scratch array's field part exactly
@pytest.mark.parametrize("L,n_sub", [(40, 4), (24, 3), (64, 4)])
def test_noalloc_diffusion_matches_context_path_twice(cuda, L, n_sub):
    torch = cuda
    from paper_2303_08123_b300 import Simulator, csr
    from paper_2303_08123_b300.sim import load_library, make_config

    lib = load_library()
    seed, step, dose = 0x5EED_00A1, 1500, 2.0
    # only the fields and the irradiation marks change: phases are long enough
    # that no cell changes kind within two steps, and cell events are off
    p = P0.replace(dur_h=(1000.0, 1000.0, 1000.0, 1000.0), flags=F_REACTION | F_DIFFUSION, n_sub=n_sub)
    fields, cell = par.random_state(L, 21, p)
    ages = np.random.default_rng(22).integers(0, 1000, L ** 3).astype(np.uint32)
    cell = np.where(cell & 7, (cell & 0xF) | (ages << 4), 0).astype(np.uint32)

    sim = Simulator([L], [-1], params=p, seed=seed)
    sim.load_protocols(*csr([([dose], [step / 600.0])]))
    sim.set_state(0, *fields, cell)
    sim.set_clock(step)
    ref = []
    for _ in range(2):
        sim.run(1)
        ref.append(sim.get_state(0))
    sim.close()

    cfg = make_config(p, seed=seed)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    dcell = torch.from_numpy(cell.view(np.int32).copy()).cuda()
    stream = torch.cuda.current_stream()
    for k, dose_k in enumerate((dose, 0.0)):  # two calls in a row: with and without a fraction
        st = lib.sim_diffuse_noalloc(ctypes.byref(cfg), L, step + k, dose_k, *(ctypes.c_void_p(t.data_ptr()) for t in dev),
                                     ctypes.c_void_p(dcell.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        O, G, H, rcell = ref[k]
        for got, want, m in zip(dev, (O, G, H), par.medium()):
            err = float(np.max(np.abs(got.cpu().numpy().astype(np.float64) - want))) / m
            assert err <= par.FIELD_TOL, (k, err)
        got_cell = dcell.cpu().numpy().view(np.uint32)
        # same kinds and DOOMED marks (the context path also aged the cells)
        assert np.array_equal(got_cell & 0xF, rcell & 0xF)
    assert np.count_nonzero(got_cell & 8) > np.count_nonzero(cell & 8)  # the fraction was applied


def test_noalloc_rejects_lattices_beyond_its_scratch(cuda):
    torch = cuda
    from paper_2303_08123_b300.sim import load_library, make_config

    lib = load_library()
    cfg = make_config(P0)
    L = 65
    bufs = [torch.zeros(L ** 3, dtype=torch.float32, device="cuda") for _ in range(3)]
    cell = torch.zeros(L ** 3, dtype=torch.int32, device="cuda")
    st = lib.sim_diffuse_noalloc(ctypes.byref(cfg), L, 0, 0.0, *(ctypes.c_void_p(t.data_ptr()) for t in bufs),
                                 ctypes.c_void_p(cell.data_ptr()), None)
    assert st == -2  # SIM_ENOSPC: larger than the fixed 64^3 scratch
    assert float(bufs[0].abs().sum()) == 0.0  # nothing was written
    bad = make_config(P0, precision="bf16")
    assert lib.sim_diffuse_noalloc(ctypes.byref(bad), 16, 0, 0.0, *(ctypes.c_void_p(t.data_ptr()) for t in bufs),
                                   ctypes.c_void_p(cell.data_ptr()), None) == -1


def test_noalloc_refuses_a_stream_under_capture(cuda):
    """The launch tables come from host memory that lives only during the call,
    so a call on a stream that is being captured is refused before any work."""
    torch = cuda
    from paper_2303_08123_b300.sim import load_library, make_config

    lib = load_library()
    cfg = make_config(P0)
    L = 16
    bufs = [torch.full((L ** 3,), 0.25, dtype=torch.float32, device="cuda") for _ in range(3)]
    cell = torch.zeros(L ** 3, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        st = lib.sim_diffuse_noalloc(ctypes.byref(cfg), L, 0, 0.0, *(ctypes.c_void_p(t.data_ptr()) for t in bufs),
                                     ctypes.c_void_p(cell.data_ptr()), ctypes.c_void_p(side.cuda_stream))
        bufs[0].add_(0.0)  # keeps the captured graph non-empty
    assert st == -1
    torch.cuda.synchronize()
    assert float(bufs[1].min()) == 0.25 and float(bufs[1].max()) == 0.25  # nothing was enqueued
