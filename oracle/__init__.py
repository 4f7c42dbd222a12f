"""FP64 CPU oracle of the EMT6/Ro spheroid CA (arxiv 2303.08123).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of the simulation that the CUDA library is checked against.  Only
the tests, the smoke check and the CPU-baseline leg of the benchmark import it;
the product path never does.  It shares no code with the CUDA library: the C
source here (oracle.c) is compiled with gcc into liboracle.so and called through
ctypes with numpy arrays.

Every function follows the model section it names in oracle.c.  Parity status:
the diffusion operator, reaction terms, irradiation, cell cycle and division are
pinned by the invariants, closed forms and brute-force checks in
tests/test_oracle_pins.py; whole-trajectory biology has no published numbers
it can be pinned to (the paper's model constants are not in the paper), so
full runs are "parity unpinned" against the paper and serve as the reference
for the CUDA path only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from synth.params import Params, STEPS_PER_HOUR

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBPATH = os.path.join(_HERE, "liboracle.so")

BC_DIRICHLET, BC_PERIODIC, BC_NOFLUX = 0, 1, 2
PURPOSE_INIT, PURPOSE_IRR, PURPOSE_DIV = 0, 1, 2
NEAR_IRR, NEAR_DEATH, NEAR_QUIESCENCE = 1, 2, 4
NEAR_TOL = 1e-5


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (the oracle is plain C: no CUDA)."""
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIBPATH
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("dur", ctypes.c_int32 * 4), ("n_sub", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("lam", ctypes.c_double * 3),
        ("medium_O", ctypes.c_double), ("medium_G", ctypes.c_double), ("medium_pH", ctypes.c_double),
        ("q_O", ctypes.c_double), ("K_O", ctypes.c_double), ("q_G", ctypes.c_double), ("K_G", ctypes.c_double),
        ("k_an", ctypes.c_double), ("O_an", ctypes.c_double), ("q_H", ctypes.c_double), ("f_Q", ctypes.c_double),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("omf_m", ctypes.c_double),
        ("omf_K", ctypes.c_double), ("phi", ctypes.c_double * 5),
        ("O_q", ctypes.c_double), ("G_q", ctypes.c_double), ("pH_q", ctypes.c_double),
        ("G_d", ctypes.c_double), ("pH_d", ctypes.c_double), ("repair_half_h", ctypes.c_double),
        ("near_tol", ctypes.c_double),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_live", "n_deaths", "n_divisions", "n_intents", "n_doomed_new", "n_decisions", "n_near")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


def _pack(p: Params, near_tol: float = NEAR_TOL) -> _Params:
    s = _Params()
    for i in range(4):
        s.dur[i] = int(round(p.dur_h[i] * STEPS_PER_HOUR))
    s.n_sub, s.flags = p.n_sub, p.flags
    for i in range(3):
        s.lam[i] = p.lam[i]
    for n in ("medium_O", "medium_G", "medium_pH", "q_O", "K_O", "q_G", "K_G", "k_an", "O_an", "q_H", "f_Q",
              "alpha", "beta", "omf_m", "omf_K", "O_q", "G_q", "pH_q", "G_d", "pH_d", "repair_half_h"):
        setattr(s, n, float(getattr(p, n)))
    for i in range(5):
        s.phi[i] = p.phi[i]
    s.near_tol = near_tol
    return s


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIBPATH)
        P = ctypes.POINTER
        u32p, f64p, i32p, i64p, u8p = P(ctypes.c_uint32), P(ctypes.c_double), P(ctypes.c_int32), \
            P(ctypes.c_int64), P(ctypes.c_uint8)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_init.restype = ctypes.c_int64
        L.or_init.argtypes = [P(_Params), ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, ctypes.c_uint32,
                              f64p, f64p, f64p, u32p]
        L.or_step.restype = ctypes.c_int
        L.or_step.argtypes = [P(_Params), ctypes.c_int, ctypes.c_int, u32p, ctypes.c_uint32, ctypes.c_uint32,
                              ctypes.c_double, ctypes.c_double, f64p, f64p, f64p, u32p, u8p, P(_Stats)]
        L.or_fraction_step.restype = ctypes.c_int64
        L.or_fraction_step.argtypes = [f64p, ctypes.c_int]
        L.or_run.restype = ctypes.c_int64
        L.or_run.argtypes = [P(_Params), ctypes.c_int, ctypes.c_int, u32p, ctypes.c_uint32, ctypes.c_uint32,
                             ctypes.c_int, f64p, f64p, ctypes.c_int64, ctypes.c_int, i32p, ctypes.c_int,
                             f64p, f64p, f64p, u32p, f64p, P(_Stats)]
        L.or_run_near.restype = ctypes.c_int64
        L.or_run_near.argtypes = L.or_run.argtypes + [u8p]
        L.or_run_batch.restype = ctypes.c_int
        L.or_run_batch.argtypes = [P(_Params), ctypes.c_int, i32p, i32p, u32p, u32p, ctypes.c_uint32, i32p,
                                   f64p, f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, i64p, i64p, i32p,
                                   ctypes.c_int, ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _key(seed: int):
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def philox(ctr, seed: int) -> np.ndarray:
    """Philox4x32-10 outputs for an (n, 4) array of uint32 counters."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    key = _key(seed)
    f = lib().or_philox4x32_10
    for i in range(ctr.shape[0]):
        f(_ptr(ctr[i], ctypes.c_uint32), _ptr(key, ctypes.c_uint32), _ptr(out[i], ctypes.c_uint32))
    return out


class State:
    """One lattice: fields O, G, H (float64, mM) and cell words (uint32), flat, index x + L(y + L z)."""

    def __init__(self, L: int):
        self.L = L
        n = L ** 3
        self.O = np.zeros(n)
        self.G = np.zeros(n)
        self.H = np.zeros(n)
        self.cell = np.zeros(n, dtype=np.uint32)

    def copy(self) -> "State":
        s = State(self.L)
        s.O[:], s.G[:], s.H[:], s.cell[:] = self.O, self.G, self.H, self.cell
        return s

    def n_live(self) -> int:
        return int(np.count_nonzero(self.cell & 7))


def init(p: Params, L: int, R: int, seed: int, init_word: int = 0xFFFFFFFF, bc: int = BC_DIRICHLET) -> State:
    st = State(L)
    pk = _pack(p)
    lib().or_init(ctypes.byref(pk), L, R, bc, _ptr(_key(seed), ctypes.c_uint32), init_word,
                  _ptr(st.O, ctypes.c_double), _ptr(st.G, ctypes.c_double), _ptr(st.H, ctypes.c_double),
                  _ptr(st.cell, ctypes.c_uint32))
    return st


def step(p: Params, st: State, seed: int, protocol: int, step_idx: int, dose: float = 0.0,
         bc: int = BC_DIRICHLET, near_tol: float = NEAR_TOL, unrepaired: float = 0.0):
    """Advance `st` in place by one CA step; returns (near flags per site, stats dict).
    `unrepaired`: dose of earlier fractions not yet repaired (incomplete-repair LQ term)."""
    pk = _pack(p, near_tol)
    near = np.zeros(st.L ** 3, dtype=np.uint8)
    stats = _Stats()
    lib().or_step(ctypes.byref(pk), st.L, bc, _ptr(_key(seed), ctypes.c_uint32), protocol, step_idx, float(dose),
                  float(unrepaired),
                  _ptr(st.O, ctypes.c_double), _ptr(st.G, ctypes.c_double), _ptr(st.H, ctypes.c_double),
                  _ptr(st.cell, ctypes.c_uint32), _ptr(near, ctypes.c_uint8), ctypes.byref(stats))
    return near, stats.as_dict()


def fraction_steps(wait_h) -> np.ndarray:
    w = np.ascontiguousarray(wait_h, dtype=np.float64)
    return np.array([lib().or_fraction_step(_ptr(w, ctypes.c_double), j) for j in range(len(w))], dtype=np.int64)


def run(p: Params, L: int, R: int, seed: int, protocol: int, doses, waits, t_end_steps: int = 0,
        regrowth_h: int = 120, hours: int = 0, init_word: int = 0xFFFFFFFF, near: bool = False):
    """Whole run from the seeded spheroid.  Returns dict(counts, state, steps, cum_dose, stats), and with
    near=True also near_any: per site the OR of the near-threshold flags of every step of the run."""
    pk = _pack(p)
    d = np.ascontiguousarray(doses, dtype=np.float64)
    w = np.ascontiguousarray(waits, dtype=np.float64)
    counts = np.full(hours + 1, -1, dtype=np.int32)
    st = State(L)
    cum = ctypes.c_double(0.0)
    tot = _Stats()
    args = (ctypes.byref(pk), L, R, _ptr(_key(seed), ctypes.c_uint32), protocol, init_word, len(d),
            _ptr(d, ctypes.c_double), _ptr(w, ctypes.c_double), int(t_end_steps), int(regrowth_h),
            _ptr(counts, ctypes.c_int32), hours, _ptr(st.O, ctypes.c_double), _ptr(st.G, ctypes.c_double),
            _ptr(st.H, ctypes.c_double), _ptr(st.cell, ctypes.c_uint32), ctypes.byref(cum), ctypes.byref(tot))
    out = {}
    if near:
        out["near_any"] = np.zeros(L ** 3, dtype=np.uint8)
        T = lib().or_run_near(*args, _ptr(out["near_any"], ctypes.c_uint8))
    else:
        T = lib().or_run(*args)
    return dict(counts=counts, state=st, steps=int(T), cum_dose=cum.value, stats=tot.as_dict(), **out)


def run_batch(p: Params, L, R, seed: int, offsets, doses, waits, p_words=None, t_end_steps: int = 0,
              regrowth_h: int = 120, max_steps: int = 0, hours: int = 0, n_threads: int = 0,
              init_word: int = 0xFFFFFFFF):
    """Many protocols, one per host thread at a time.  Returns dict(n_final, steps, counts)."""
    pk = _pack(p)
    L = np.ascontiguousarray(L, dtype=np.int32)
    R = np.ascontiguousarray(R, dtype=np.int32)
    n = len(L)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    d = np.ascontiguousarray(doses, dtype=np.float64)
    w = np.ascontiguousarray(waits, dtype=np.float64)
    pw = np.arange(n, dtype=np.uint32) if p_words is None else np.ascontiguousarray(p_words, dtype=np.uint32)
    n_final = np.zeros(n, dtype=np.int64)
    steps = np.zeros(n, dtype=np.int64)
    counts = np.full(n * (hours + 1), -1, dtype=np.int32)
    if n_threads <= 0:
        n_threads = os.cpu_count() or 1
    if len(d) == 0:
        d = np.zeros(1)
        w = np.zeros(1)
    lib().or_run_batch(ctypes.byref(pk), n, _ptr(L, ctypes.c_int32), _ptr(R, ctypes.c_int32),
                       _ptr(_key(seed), ctypes.c_uint32), _ptr(pw, ctypes.c_uint32), init_word,
                       _ptr(off, ctypes.c_int32), _ptr(d, ctypes.c_double), _ptr(w, ctypes.c_double),
                       int(t_end_steps), int(regrowth_h), int(max_steps), _ptr(n_final, ctypes.c_int64),
                       _ptr(steps, ctypes.c_int64), _ptr(counts, ctypes.c_int32), hours, n_threads)
    return dict(n_final=n_final, steps=steps, counts=counts.reshape(n, hours + 1))
