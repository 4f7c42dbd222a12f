"""Python binding of libsim (include/sim.h): argument marshalling only.

Every step of the simulation runs in the CUDA library; this module converts
numpy arrays to pointers, allocates the device workspace with PyTorch and
passes PyTorch's CUDA stream.  If the library is not built, `load_library`
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from synth.params import P0, Params, STEPS_PER_HOUR

_LIBDIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib")

SIM_FP32, SIM_BF16, SIM_FP16 = 0, 1, 2
_PRECISION = {"fp32": SIM_FP32, "bf16": SIM_BF16, "fp16": SIM_FP16}


class SimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libsim status {status}: {msg}")
        self.status = status


class SimParams(ctypes.Structure):
    _fields_ = [
        ("dur_h", ctypes.c_double * 4), ("n_sub", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("lam", ctypes.c_double * 3),
        ("medium_O", ctypes.c_double), ("medium_G", ctypes.c_double), ("medium_pH", ctypes.c_double),
        ("q_O", ctypes.c_double), ("K_O", ctypes.c_double), ("q_G", ctypes.c_double), ("K_G", ctypes.c_double),
        ("k_an", ctypes.c_double), ("O_an", ctypes.c_double), ("q_H", ctypes.c_double), ("f_Q", ctypes.c_double),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("omf_m", ctypes.c_double),
        ("omf_K", ctypes.c_double), ("phi", ctypes.c_double * 5),
        ("O_q", ctypes.c_double), ("G_q", ctypes.c_double), ("pH_q", ctypes.c_double),
        ("G_d", ctypes.c_double), ("pH_d", ctypes.c_double), ("repair_half_h", ctypes.c_double),
    ]


class SimConfig(ctypes.Structure):
    _fields_ = [
        ("params", SimParams), ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
        ("regrowth_h", ctypes.c_int32), ("t_end_steps", ctypes.c_int64), ("n_max_fitness", ctypes.c_double),
        ("dose_cap_gy", ctypes.c_double), ("hours", ctypes.c_int32), ("max_fractions", ctypes.c_int32),
        ("init_word", ctypes.c_uint32), ("use_graphs", ctypes.c_int32), ("path", ctypes.c_int32),
        ("tile_shape", ctypes.c_int32), ("z_chunk", ctypes.c_int32),
    ]


def pack_params(p: Params) -> SimParams:
    s = SimParams()
    for i in range(4):
        s.dur_h[i] = p.dur_h[i]
    s.n_sub, s.flags = p.n_sub, p.flags
    for i in range(3):
        s.lam[i] = p.lam[i]
    for n in ("medium_O", "medium_G", "medium_pH", "q_O", "K_O", "q_G", "K_G", "k_an", "O_an", "q_H", "f_Q",
              "alpha", "beta", "omf_m", "omf_K", "O_q", "G_q", "pH_q", "G_d", "pH_d", "repair_half_h"):
        setattr(s, n, float(getattr(p, n)))
    for i in range(5):
        s.phi[i] = p.phi[i]
    return s


_lib = None

# exported symbols and their signatures (restype, argtypes)
_P = ctypes.POINTER
_vp, _i32p, _u32p, _f32p, _f64p, _i64p = ctypes.c_void_p, _P(ctypes.c_int32), _P(ctypes.c_uint32), \
    _P(ctypes.c_float), _P(ctypes.c_double), _P(ctypes.c_int64)
SIGNATURES = {
    "sim_workspace_size": (ctypes.c_int, [_P(SimConfig), ctypes.c_int, _i32p, _P(ctypes.c_size_t)]),
    "sim_create": (ctypes.c_int, [_P(SimConfig), ctypes.c_int, _i32p, _i32p, _vp, ctypes.c_size_t, _vp,
                                  _P(_vp)]),
    "sim_load_protocols": (ctypes.c_int, [_vp, ctypes.c_int, _i32p, _f64p, _f64p]),
    "sim_reset": (ctypes.c_int, [_vp]),
    "sim_load_dose_vectors": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_double]),
    "sim_fitness_device": (ctypes.c_int, [_vp, _vp, _vp]),
    "sim_run": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "sim_fitness": (ctypes.c_int, [_vp, _i32p, _f64p]),
    "sim_counts": (ctypes.c_int, [_vp, _i32p, ctypes.c_int]),
    "sim_delivered_dose": (ctypes.c_int, [_vp, _f64p]),
    "sim_field_totals": (ctypes.c_int, [_vp, _f64p, _f32p]),
    "sim_clock": (ctypes.c_int, [_vp, _i64p, _i64p]),
    "sim_set_clock": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "sim_get_state": (ctypes.c_int, [_vp, ctypes.c_int, _f32p, _f32p, _f32p, _u32p]),
    "sim_set_state": (ctypes.c_int, [_vp, ctypes.c_int, _f32p, _f32p, _f32p, _u32p]),
    "sim_copy_lattice": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int]),
    "sim_save_state": (ctypes.c_int, [_vp, _vp, _P(ctypes.c_size_t)]),
    "sim_load_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "sim_profile_steps": (ctypes.c_int, [_vp, ctypes.c_int, _f64p, _i64p]),
    "sim_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _P(ctypes.c_int), _f64p]),
    "sim_diffuse_noalloc": (ctypes.c_int, [_P(SimConfig), ctypes.c_int, ctypes.c_int64, ctypes.c_double, _vp, _vp,
                                           _vp, _vp, _vp]),
    "sim_last_error": (ctypes.c_char_p, [_vp]),
    "sim_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sim_destroy": (None, [_vp]),
}


def library_path(check: bool = False) -> str:
    return os.path.join(_LIBDIR, "libsim_check.so" if check else "libsim.so")


_check_lib = None


def load_library(check: bool = False) -> ctypes.CDLL:
    """Load libsim.so (check=True: the index-checking debug build libsim_check.so);
    raises if it has not been built (no fallback exists)."""
    global _lib, _check_lib
    if (_check_lib if check else _lib) is None:
        path = library_path(check)
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2303_08123_b300._build` "
                               "(the simulator has no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        if check:
            _check_lib = lib
        else:
            _lib = lib
    return _check_lib if check else _lib


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def make_config(params: Params = P0, seed: int = 0x5EED, precision="fp32", regrowth_h: int = 120,
                t_end_steps: int = 0, n_max_fitness: float = 1500.0, dose_cap_gy: float = 30.0,
                hours: int = 0, max_fractions: int = 240, init_word: int = 0xFFFFFFFF,
                use_graphs: bool = True, path: str = "fused", tile_shape: int = 0, z_chunk: int = 0) -> SimConfig:
    c = SimConfig()
    c.params = pack_params(params)
    c.seed = seed
    c.precision = _PRECISION[precision] if isinstance(precision, str) else int(precision)
    c.regrowth_h = regrowth_h
    c.t_end_steps = t_end_steps
    c.n_max_fitness = n_max_fitness
    c.dose_cap_gy = dose_cap_gy
    c.hours = hours
    c.max_fractions = max_fractions
    c.init_word = init_word
    c.use_graphs = int(use_graphs)
    c.path = {"fused": 0, "substep": 1}[path] if isinstance(path, str) else int(path)
    c.tile_shape = tile_shape
    c.z_chunk = z_chunk
    return c


class Simulator:
    """A batch of protocol slots on one GPU (one libsim context).

    L, R: lattice size and initial spheroid radius per slot.  The workspace is
    a PyTorch uint8 tensor on `device`; work runs on `stream` (default: the
    current PyTorch stream).  check=True runs the index-checking debug build
    (a kernel that addresses a site outside the batch skips the access and the
    next synchronising call raises).
    """

    def __init__(self, L, R, config: SimConfig | None = None, device="cuda", stream=None, check: bool = False,
                 **cfg_kw):
        import torch

        self._lib = load_library(check)
        self.L = np.ascontiguousarray(L, dtype=np.int32)
        self.R = np.ascontiguousarray(R, dtype=np.int32)
        self.n = len(self.L)
        self.config = config if config is not None else make_config(**cfg_kw)
        size = ctypes.c_size_t(0)
        self._check(self._lib.sim_workspace_size(ctypes.byref(self.config), self.n, _ptr(self.L, ctypes.c_int32),
                                                 ctypes.byref(size)), None)
        self.workspace_bytes = size.value
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        ctx = ctypes.c_void_p()
        self._check(self._lib.sim_create(ctypes.byref(self.config), self.n, _ptr(self.L, ctypes.c_int32),
                                         _ptr(self.R, ctypes.c_int32), ctypes.c_void_p(self.workspace.data_ptr()),
                                         size.value, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx)),
                    None)
        self._ctx = ctx

    # ------------------------------------------------------------------ plumbing
    def _check(self, status, ctx):
        if status != 0:
            msg = self._lib.sim_last_error(ctx).decode() if ctx else ""
            raise SimError(status, msg or self._lib.sim_status_string(status).decode())

    def _call(self, name, *args):
        self._check(getattr(self._lib, name)(self._ctx, *args), self._ctx)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.sim_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ API
    def load_protocols(self, offsets, doses, waits):
        off = np.ascontiguousarray(offsets, dtype=np.int32)
        d = np.ascontiguousarray(doses, dtype=np.float64)
        w = np.ascontiguousarray(waits, dtype=np.float64)
        self._call("sim_load_protocols", self.n, _ptr(off, ctypes.c_int32), _ptr(d, ctypes.c_double),
                   _ptr(w, ctypes.c_double))

    def reset(self):
        self._call("sim_reset")

    def run(self, max_steps: int = 0):
        self._call("sim_run", int(max_steps))

    def load_dose_vectors(self, units, unit_gy: float = 0.25):
        """Protocols from a device uint8 tensor [n, n_slots] of dose units per
        30-min slot (asynchronous; keep `units` alive until the stream passes)."""
        import torch
        if not (units.is_cuda and units.dtype == torch.uint8 and units.dim() == 2 and units.is_contiguous()
                and units.shape[0] == self.n):
            raise ValueError("units must be a contiguous CUDA uint8 tensor of shape [n_protocols, n_slots]")
        self._call("sim_load_dose_vectors", ctypes.c_void_p(units.data_ptr()), int(units.shape[1]), float(unit_gy))

    def fitness_device(self, count=None, fitness=None):
        """Final counts (int32) and fitness n_max - n (float32) into device
        tensors on the stream, without synchronising; returns (count, fitness)."""
        import torch
        dev = self.workspace.device
        count = torch.empty(self.n, dtype=torch.int32, device=dev) if count is None else count
        fitness = torch.empty(self.n, dtype=torch.float32, device=dev) if fitness is None else fitness
        self._call("sim_fitness_device", ctypes.c_void_p(count.data_ptr()), ctypes.c_void_p(fitness.data_ptr()))
        return count, fitness

    def fitness(self):
        cnt = np.zeros(self.n, dtype=np.int32)
        fit = np.zeros(self.n, dtype=np.float64)
        self._call("sim_fitness", _ptr(cnt, ctypes.c_int32), _ptr(fit, ctypes.c_double))
        return cnt, fit

    def counts(self):
        h = self.config.hours
        out = np.zeros(self.n * (h + 1), dtype=np.int32)
        self._call("sim_counts", _ptr(out, ctypes.c_int32), h)
        return out.reshape(self.n, h + 1)

    def field_totals(self):
        """(FP64 totals, Kahan FP32 totals), each n x 3 (O2, glucose, H+) in mM summed over sites."""
        a = np.zeros(self.n * 3, dtype=np.float64)
        b = np.zeros(self.n * 3, dtype=np.float32)
        self._call("sim_field_totals", _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_float))
        return a.reshape(self.n, 3), b.reshape(self.n, 3)

    def delivered_dose(self):
        out = np.zeros(self.n, dtype=np.float64)
        self._call("sim_delivered_dose", _ptr(out, ctypes.c_double))
        return out

    def clock(self):
        st = np.zeros(self.n, dtype=np.int64)
        te = np.zeros(self.n, dtype=np.int64)
        self._call("sim_clock", _ptr(st, ctypes.c_int64), _ptr(te, ctypes.c_int64))
        return st, te

    def set_clock(self, step: int):
        self._call("sim_set_clock", int(step))

    def get_state(self, p: int):
        n = int(self.L[p]) ** 3
        O, G, H = (np.zeros(n, dtype=np.float32) for _ in range(3))
        cell = np.zeros(n, dtype=np.uint32)
        self._call("sim_get_state", p, _ptr(O, ctypes.c_float), _ptr(G, ctypes.c_float), _ptr(H, ctypes.c_float),
                   _ptr(cell, ctypes.c_uint32))
        return O, G, H, cell

    def set_state(self, p: int, O, G, H, cell):
        f = [np.ascontiguousarray(a, dtype=np.float32) for a in (O, G, H)]
        c = np.ascontiguousarray(cell, dtype=np.uint32)
        self._call("sim_set_state", p, *(_ptr(a, ctypes.c_float) for a in f), _ptr(c, ctypes.c_uint32))

    def profile_steps(self, n_steps: int):
        """Advance n_steps plain steps; per-kernel-class device ms and launch counts
        (substep, cell, claim, resolve)."""
        ms = np.zeros(4, dtype=np.float64)
        nl = np.zeros(4, dtype=np.int64)
        self._call("sim_profile_steps", int(n_steps), _ptr(ms, ctypes.c_double), _ptr(nl, ctypes.c_int64))
        return ms, nl

    def autotune(self, n_steps: int = 10):
        """Time every fused tile shape on this batch, keep the fastest and re-seed
        the batch at step 0.  Returns (best shape, ms per step per shape)."""
        best = ctypes.c_int(0)
        ms = np.full(8, -1.0)
        self._call("sim_autotune", int(n_steps), ctypes.byref(best), _ptr(ms, ctypes.c_double))
        return best.value, ms

    def copy_lattice(self, p: int, src: "Simulator", q: int):
        """Slot p of this batch <- slot q of `src` (device to device)."""
        self._call("sim_copy_lattice", p, src._ctx, q)

    def save_state(self) -> bytes:
        size = ctypes.c_size_t(0)
        self._call("sim_save_state", None, ctypes.byref(size))
        buf = ctypes.create_string_buffer(size.value)
        self._call("sim_save_state", ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(size))
        return buf.raw[:size.value]

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._call("sim_load_state", ctypes.cast(buf, ctypes.c_void_p), len(blob))


def csr(protocols):
    """[(doses, waits), ...] -> (offsets, doses, waits) CSR arrays."""
    off = [0]
    d, w = [], []
    for dd, ww in protocols:
        d.extend(dd)
        w.extend(ww)
        off.append(len(d))
    return np.array(off, dtype=np.int32), np.array(d, dtype=np.float64), np.array(w, dtype=np.float64)


__all__ = ["Simulator", "SimError", "make_config", "load_library", "csr", "SIGNATURES", "STEPS_PER_HOUR"]
