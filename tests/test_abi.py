"""C ABI checks that need no GPU: the library loads, exports every entry point
the headers declare, has the struct layout the binding assumes, and rejects
bad configurations before touching a device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z]+_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_08123_b300 import _build
    _build.build()
    from paper_2303_08123_b300.sim import load_library
    return load_library()


def test_every_declared_symbol_is_exported(lib):
    from paper_2303_08123_b300.sim import SIGNATURES
    names = declared("sim.h")
    assert {"sim_create", "sim_run", "sim_fitness", "sim_load_protocols"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
        assert n in SIGNATURES, f"binding lacks {n}"


def test_workspace_size_validation(lib):
    from paper_2303_08123_b300.sim import make_config
    from synth.params import P0

    cfg = make_config(P0, hours=10)
    size = ctypes.c_size_t()
    L = np.array([40, 64], dtype=np.int32)
    Lp = L.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    assert lib.sim_workspace_size(ctypes.byref(cfg), 2, Lp, ctypes.byref(size)) == 0
    # 2 x 3 FP32 fields (24) + 2 cell words (8) + claim (8) + work list (8) = 48 B per site, plus tables
    sites = 40 ** 3 + 64 ** 3
    assert 48 * sites <= size.value <= 48 * sites + 2_000_000
    bad = np.array([7], dtype=np.int32)
    assert lib.sim_workspace_size(ctypes.byref(cfg), 1, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  ctypes.byref(size)) == -1
    assert lib.sim_workspace_size(ctypes.byref(cfg), 0, Lp, ctypes.byref(size)) == -1
    unstable = make_config(P0.replace(lam=(0.2, 0.05, 0.1)))
    assert lib.sim_workspace_size(ctypes.byref(unstable), 2, Lp, ctypes.byref(size)) == -1
    for bad_params in (P0.replace(repair_half_h=-1.0), P0.replace(repair_half_h=float("nan")),
                       P0.replace(n_sub=0), P0.replace(n_sub=257)):
        cfg_bad = make_config(bad_params)
        assert lib.sim_workspace_size(ctypes.byref(cfg_bad), 2, Lp, ctypes.byref(size)) == -1
    assert lib.sim_workspace_size(ctypes.byref(make_config(P0.replace(n_sub=256))), 2, Lp, ctypes.byref(size)) == 0
    half = make_config(P0, precision="bf16", hours=10)
    s2 = ctypes.c_size_t()
    assert lib.sim_workspace_size(ctypes.byref(half), 2, Lp, ctypes.byref(s2)) == 0
    assert s2.value < size.value  # 2-byte field storage


def test_null_context_calls_are_rejected(lib):
    assert lib.sim_run(None, 1) == -1
    assert lib.sim_fitness(None, None, None) == -1
    lib.sim_destroy(None)  # no-op
    assert lib.sim_status_string(-4) == b"device wait timed out"


def test_binding_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors of sim_params / sim_config have the C layout."""
    from paper_2303_08123_b300.sim import SimConfig, SimParams
    fields = [f for f, _ in SimConfig._fields_]
    pf = [f for f, _ in SimParams._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sim.h"', 'int main(void){',
             'printf("%zu %zu\\n", sizeof(sim_config), sizeof(sim_params));']
    lines += [f'printf("%zu\\n", offsetof(sim_config, {f}));' for f in fields]
    lines += [f'printf("%zu\\n", offsetof(sim_params, {f}));' for f in pf]
    lines += ["return 0;}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).decode().split()]
    assert vals[0] == ctypes.sizeof(SimConfig) and vals[1] == ctypes.sizeof(SimParams)
    assert vals[2:2 + len(fields)] == [getattr(SimConfig, f).offset for f in fields]
    assert vals[2 + len(fields):] == [getattr(SimParams, f).offset for f in pf]


def test_mlp_library_exports_every_declared_symbol():
    from paper_2303_08123_b300 import _build
    _build.build()
    from paper_2303_08123_b300.surrogate import SIGNATURES, load_library
    lib = load_library()
    names = declared("mlp.h")
    assert {"mlp_create", "mlp_forward", "mlp_train_step", "mlp_gradients", "mlp_gemm_bf16"} <= set(names)
    for n in names:
        assert hasattr(lib, n) and n in SIGNATURES, n
    assert lib.mlp_num_params() == 256 * 48 + 256 + 2 * (256 * 256 + 256) + 256 + 1
    size = ctypes.c_size_t()
    assert lib.mlp_workspace_size(100, ctypes.byref(size)) == -1  # batches are multiples of 128
    assert lib.mlp_workspace_size(256, ctypes.byref(size)) == 0 and size.value > 0


def test_ga_library_exports_and_layout(tmp_path):
    """libga exports what ga.h declares, the binding mirrors ga_params, and bad
    arguments are rejected before any device work."""
    from paper_2303_08123_b300 import _build
    _build.build()
    from paper_2303_08123_b300.devga import SIGNATURES, GaParams, load_library, make_params
    lib = load_library()
    for n in declared("ga.h"):
        assert hasattr(lib, n) and n in SIGNATURES, n
    fields = [f for f, _ in GaParams._fields_]
    src = tmp_path / "ga_layout.c"
    src.write_text("\n".join(['#include <stdio.h>', '#include <stddef.h>', '#include "ga.h"', 'int main(void){',
                              'printf("%zu\\n", sizeof(ga_params));']
                             + [f'printf("%zu\\n", offsetof(ga_params, {f}));' for f in fields] + ["return 0;}"]))
    exe = tmp_path / "ga_layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).decode().split()]
    assert vals == [ctypes.sizeof(GaParams)] + [getattr(GaParams, f).offset for f in fields]
    size = ctypes.c_size_t()
    assert lib.ga_workspace_size(0, ctypes.byref(size)) == -1
    assert lib.ga_workspace_size(4096, ctypes.byref(size)) == 0 and size.value >= 16 * 4096
    ok = make_params()
    for bad in (dict(n_slots=0), dict(n_slots=2000), dict(d_max=0), dict(min_gap=0), dict(n_parents=0),
                dict(selection=3), dict(crossover=7), dict(mutations=16), dict(p_mut=1.5),
                dict(selection=2, tournament_k=65)):
        p = make_params(**bad)
        assert lib.ga_random_population(ctypes.byref(p), 64, 1, ctypes.c_void_p(1), None) == -1, bad
    assert lib.ga_generation(ctypes.byref(ok), 64, None, None, 1, 0, None, None, None, 0, None) == -1
