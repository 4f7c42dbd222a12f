"""Python binding of libga (include/ga.h): the paper's GA operators run on the
device, so that a GA loop over the batched simulator never leaves the GPU.
Argument marshalling only; every operator runs in the CUDA library.

    DeviceGA(params, P)                 one population size, scratch on the GPU
      .random_population(seed)          uint8 [P, S] dose units per 30-min slot
      .generation(pop, fitness, seed, g) next population (elites first) and ranking
    params_from_config(cfg, P)          ga_params from the host GA's GAConfig
    evolve_on_device(sim, dga, ...)     whole GA loop: simulate, score, breed, on the stream
"""
from __future__ import annotations

import ctypes
import os

from .sim import SimError

_LIBDIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib")
_lib = None
_vp = ctypes.c_void_p

SEL = {"simple": 0, "roulette": 1, "tournament": 2}
CROSS = {"single_point": 0, "two_point": 1, "uniform": 2}
MUT = {"swap": 1, "split": 2, "dose_time": 4, "dose_value": 8}


class GaParams(ctypes.Structure):
    _fields_ = [
        ("n_slots", ctypes.c_int32), ("d_max", ctypes.c_int32), ("total_cap", ctypes.c_int32),
        ("min_gap", ctypes.c_int32), ("n_elite", ctypes.c_int32), ("n_parents", ctypes.c_int32),
        ("selection", ctypes.c_int32), ("crossover", ctypes.c_int32), ("mutations", ctypes.c_uint32),
        ("p_mut", ctypes.c_float), ("tournament_k", ctypes.c_int32), ("tournament_q", ctypes.c_float),
    ]


SIGNATURES = {
    "ga_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "ga_random_population": (ctypes.c_int, [ctypes.POINTER(GaParams), ctypes.c_int, ctypes.c_uint64, _vp, _vp]),
    "ga_generation": (ctypes.c_int, [ctypes.POINTER(GaParams), ctypes.c_int, _vp, _vp, ctypes.c_uint64,
                                     ctypes.c_uint32, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
}


def load_library() -> ctypes.CDLL:
    """Load libga.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        path = os.path.join(_LIBDIR, "libga.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2303_08123_b300._build`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        _lib = lib
    return _lib


def make_params(n_slots=240, d_max=8, total_cap=40, min_gap=12, n_elite=4, n_parents=16, selection=0, crossover=1,
                mutations=1 | 2 | 4, p_mut=0.3, tournament_k=16, tournament_q=0.9) -> GaParams:
    p = GaParams()
    for k, v in dict(n_slots=n_slots, d_max=d_max, total_cap=total_cap, min_gap=min_gap, n_elite=n_elite,
                     n_parents=n_parents, selection=selection, crossover=crossover, mutations=mutations,
                     p_mut=p_mut, tournament_k=tournament_k, tournament_q=tournament_q).items():
        setattr(p, k, v)
    return p


def params_from_config(cfg, P: int, unit_gy: float = 0.25) -> GaParams:
    """ga_params equivalent to the host GA's GAConfig (doses in units of unit_gy)."""
    mut = 0
    for m in cfg.mutations:
        mut |= MUT[m]
    return make_params(n_slots=cfg.n_slots, d_max=int(round(cfg.d_max / unit_gy)),
                       total_cap=int(round(cfg.total_cap / unit_gy)), min_gap=cfg.min_gap,
                       n_elite=max(1, int(round(cfg.elite_frac * P))), n_parents=max(2, int(round(cfg.parent_frac * P))),
                       selection=SEL[cfg.selection], crossover=CROSS[cfg.crossover], mutations=mut, p_mut=cfg.p_mut,
                       tournament_k=min(cfg.tournament_k, P), tournament_q=cfg.tournament_q)


class DeviceGA:
    """GA operators for populations of P dose vectors on one CUDA device."""

    def __init__(self, params: GaParams, P: int, device="cuda", stream=None):
        import torch

        self._lib = load_library()
        self.params, self.P = params, int(P)
        size = ctypes.c_size_t(0)
        self._check(self._lib.ga_workspace_size(self.P, ctypes.byref(size)))
        self.workspace = torch.empty(max(1, size.value), dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)

    @staticmethod
    def _check(status):
        if status != 0:
            raise SimError(status, "libga call failed")

    def _empty_pop(self):
        import torch
        return torch.empty((self.P, self.params.n_slots), dtype=torch.uint8, device=self.workspace.device)

    def random_population(self, seed: int, out=None):
        out = self._empty_pop() if out is None else out
        self._check(self._lib.ga_random_population(ctypes.byref(self.params), self.P, seed,
                                                   _vp(out.data_ptr()), _vp(self.stream.cuda_stream)))
        return out

    def generation(self, pop, fitness, seed: int, gen: int, out=None, order=None):
        """Next population from `pop` (uint8 [P, S]) under `fitness` (float32 [P],
        higher is better); returns (next, ranking)."""
        import torch
        out = self._empty_pop() if out is None else out
        order = torch.empty(self.P, dtype=torch.int32, device=pop.device) if order is None else order
        for t, dt in ((pop, torch.uint8), (fitness, torch.float32), (out, torch.uint8), (order, torch.int32)):
            if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
                raise ValueError("pop/out must be contiguous CUDA uint8, fitness float32, order int32")
        self._check(self._lib.ga_generation(ctypes.byref(self.params), self.P, _vp(pop.data_ptr()),
                                            _vp(fitness.data_ptr()), seed, gen, _vp(out.data_ptr()),
                                            _vp(order.data_ptr()), _vp(self.workspace.data_ptr()),
                                            self.workspace.numel(), _vp(self.stream.cuda_stream)))
        return out, order


def evolve_on_device(sim, dga: DeviceGA, generations: int, seed: int, unit_gy: float = 0.25, pop=None):
    """The paper's main GA loop with every step on the device: load the
    population's dose vectors into the simulator, run every protocol to the
    fixed horizon, score (fitness = n_max - final count), breed the next
    population.  The host only enqueues work (the simulator synchronises only
    when its work list changes, which a fixed horizon never causes); nothing is
    read back until the caller reads the results.  Returns (final population,
    fitness history tensor [generations + 1, P] on the device)."""
    import torch

    pop = dga.random_population(seed) if pop is None else pop
    spare = torch.empty_like(pop)
    hist = torch.empty((generations + 1, dga.P), dtype=torch.float32, device=pop.device)
    for g in range(generations + 1):
        sim.load_dose_vectors(pop, unit_gy)
        sim.run(0)
        _, fit = sim.fitness_device(fitness=hist[g])
        if g == generations:
            break
        pop, spare = dga.generation(pop, fit, seed, g + 1, out=spare)[0], pop
    return pop, hist


def main():
    """Time one device GA generation at the paper-scale population (4,096 dose
    vectors of 240 half-hour slots) for each selection scheme; one JSON line each."""
    import json

    import torch

    P = 4096
    for sel in ("simple", "roulette", "tournament"):
        prm = make_params(n_slots=240, d_max=8, total_cap=40, min_gap=12, n_elite=410, n_parents=1638,
                          selection=SEL[sel], crossover=CROSS["two_point"], mutations=15, p_mut=0.3)
        dga = DeviceGA(prm, P)
        pop = dga.random_population(7)
        fit = torch.rand(P, device=pop.device)
        out = torch.empty_like(pop)
        for _ in range(3):
            dga.generation(pop, fit, 7, 1, out=out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(dga.stream)
        n = 20
        for g in range(n):
            dga.generation(pop, fit, 7, g, out=out)
        b.record(dga.stream)
        torch.cuda.synchronize()
        print(json.dumps({"selection": sel, "population": P, "slots": 240,
                          "ms_per_generation": a.elapsed_time(b) / n}))


if __name__ == "__main__":
    main()
