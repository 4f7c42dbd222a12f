"""Python binding of libmlp (include/mlp.h): the surrogate network that
pre-screens GA candidates.  Argument marshalling only; the forward pass,
backward pass and optimiser run in the CUDA library on the tensor cores."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .sim import SimError

_LIBDIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib")
_lib = None
_P = ctypes.POINTER
_vp = ctypes.c_void_p
SIGNATURES = {
    "mlp_num_params": (ctypes.c_int, []),
    "mlp_workspace_size": (ctypes.c_int, [ctypes.c_int, _P(ctypes.c_size_t)]),
    "mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, _vp, ctypes.c_size_t, _vp, _P(_vp)]),
    "mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "mlp_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _P(ctypes.c_float)]),
    "mlp_gradients": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _P(ctypes.c_float)]),
    "mlp_get_params": (ctypes.c_int, [_vp, _P(ctypes.c_float)]),
    "mlp_set_params": (ctypes.c_int, [_vp, _P(ctypes.c_float)]),
    "mlp_gemm_bf16": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "mlp_wait_probe": (ctypes.c_int, [ctypes.c_uint32, _vp, _vp]),
    "mlp_destroy": (None, [_vp]),
}


def load_library() -> ctypes.CDLL:
    """Load libmlp.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        path = os.path.join(_LIBDIR, "libmlp.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2303_08123_b300._build`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        _lib = lib
    return _lib


def _check(status):
    if status != 0:
        raise SimError(status, "libmlp call failed")


def gemm_bf16(A, B):
    """C = A B^T on the tensor cores (torch BF16 CUDA tensors, row-major)."""
    import torch
    lib = load_library()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty(M, N, dtype=torch.float32, device=A.device)
    st = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.mlp_gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, st.data_ptr(),
                             torch.cuda.current_stream(A.device).cuda_stream))
    torch.cuda.synchronize(A.device)
    if int(st.item()) != 0:
        raise SimError(-4, "tensor-core GEMM timed out")
    return C


class Surrogate:
    """45 -> 256 -> 256 -> 256 -> 1 GELU network with tensor-core training."""

    def __init__(self, batch_max: int = 4096, seed: int = 7, device="cuda"):
        import torch
        self._lib = load_library()
        self.batch_max = batch_max
        self.n_params = self._lib.mlp_num_params()
        size = ctypes.c_size_t()
        _check(self._lib.mlp_workspace_size(batch_max, ctypes.byref(size)))
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=device)
        self.device = self.workspace.device
        self.stream = torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p()
        _check(self._lib.mlp_create(batch_max, seed, self.workspace.data_ptr(), size.value, self.stream.cuda_stream,
                                    ctypes.byref(ctx)))
        self._ctx = ctx

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.mlp_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(self.device)

    def forward(self, X):
        import torch
        Xd = X if hasattr(X, "data_ptr") else self._dev(X)
        y = torch.empty(Xd.shape[0], dtype=torch.float32, device=self.device)
        _check(self._lib.mlp_forward(self._ctx, Xd.data_ptr(), Xd.shape[0], y.data_ptr()))
        return y

    def predict(self, X) -> np.ndarray:
        """Forward over any number of rows (padded to batches of 128)."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        n = X.shape[0]
        out = np.empty(n, dtype=np.float32)
        for s in range(0, n, self.batch_max):
            chunk = X[s:s + self.batch_max]
            m = chunk.shape[0]
            pad = (-m) % 128
            if pad:
                chunk = np.concatenate([chunk, np.zeros((pad, X.shape[1]), dtype=np.float32)])
            out[s:s + m] = self.forward(chunk).cpu().numpy()[:m]
        return out

    def train_step(self, X, t, lr: float, want_loss: bool = True):
        """One Adam step; returns the loss before the step (synchronises), or None
        without synchronising when want_loss is False."""
        Xd = X if hasattr(X, "data_ptr") else self._dev(X)
        td = t if hasattr(t, "data_ptr") else self._dev(t)
        loss = ctypes.c_float()
        _check(self._lib.mlp_train_step(self._ctx, Xd.data_ptr(), td.data_ptr(), Xd.shape[0], float(lr),
                                        ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def gradients(self, X, t):
        import torch
        Xd, td = self._dev(X), self._dev(t)
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        loss = ctypes.c_float()
        _check(self._lib.mlp_gradients(self._ctx, Xd.data_ptr(), td.data_ptr(), Xd.shape[0], g.data_ptr(),
                                       ctypes.byref(loss)))
        return g.cpu().numpy(), loss.value

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(self._lib.mlp_get_params(self._ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.mlp_set_params(self._ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))


def main():
    """Time the network on the tensor cores at the largest batch: forward and
    one training step (forward, backward, Adam) over 4,096 rows; one JSON line."""
    import json

    import torch

    B, n = 4096, 50
    net = Surrogate(batch_max=B, seed=1)
    X = torch.rand(B, 45, device=net.device)
    t = torch.rand(B, device=net.device)
    fwd_flop = 2.0 * B * (48 * 256 + 2 * 256 * 256 + 256)
    out = {"batch": B}
    for name, fn, flop in (("forward", lambda: net.forward(X), fwd_flop),
                           ("train_step", lambda: net.train_step(X, t, 1e-4, want_loss=False), 3 * fwd_flop)):
        for _ in range(5):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(net.stream)
        for _ in range(n):
            fn()
        b.record(net.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n
        out[name] = {"ms": ms, "gemm_tflops": flop / (ms / 1e3) / 1e12}
    # one GEMM at the network's widths over many rows: what the tensor-core kernel sustains when it has work
    lib = load_library()
    M, N, K = 65536, 256, 256
    A = torch.randn(M, K, device=net.device).to(torch.bfloat16)
    Bm = torch.randn(N, K, device=net.device).to(torch.bfloat16)
    C = torch.empty(M, N, dtype=torch.float32, device=net.device)
    st = torch.zeros(1, dtype=torch.int32, device=net.device)
    call = lambda: lib.mlp_gemm_bf16(A.data_ptr(), Bm.data_ptr(), C.data_ptr(), M, N, K, st.data_ptr(),  # noqa: E731
                                     net.stream.cuda_stream)
    for _ in range(5):
        _check(call())
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(net.stream)
    for _ in range(n):
        call()
    b.record(net.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    out["gemm_65536x256x256"] = {"ms": ms, "tflops": 2.0 * M * N * K / (ms / 1e3) / 1e12,
                                 "status": int(st.item())}
    print(json.dumps(out))


if __name__ == "__main__":
    main()

