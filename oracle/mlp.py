"""FP64 reference of the surrogate network (test infrastructure only).

The plain definition of the network in numpy: 45 inputs (zero-padded to 48),
three hidden layers of 256 with GELU (erf form), one linear output, mean
squared error.  The CUDA library feeds the tensor cores BF16 operands; with
`bf16=True` this reference rounds the same tensors to BF16 (round to nearest
even) at the same points, so gradients can be compared tightly.  Parameter
vector order: W1 (256 x 48), b1, W2 (256 x 256), b2, W3, b3, w4 (256), b4.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

H, IP, IN = 256, 48, 45
SHAPES = [("W1", (H, IP)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("w4", (H,)), ("b4", (1,))]


def unpack(p):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def to_bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(p, X, bf16=True):
    """Returns (y, cache)."""
    P = unpack(p)
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.zeros((X.shape[0], IP))
    x[:, :IN] = X
    a = r(x)
    cache = {"a": [a], "z": []}
    for l, (W, b) in enumerate((("W1", "b1"), ("W2", "b2"), ("W3", "b3"))):
        z = a @ r(P[W]).T + P[b]
        h = gelu(z)
        cache["z"].append(z)
        cache["h_last"] = h
        a = r(h)
        cache["a"].append(a)
    y = cache["h_last"] @ P["w4"] + P["b4"][0]
    return y, cache


def gradients(p, X, t, bf16=True):
    """Gradient of mean((y - t)^2) with respect to the parameter vector; returns (grad, loss)."""
    P = unpack(p)
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(p, X, bf16)
    B = X.shape[0]
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B
    g = {"w4": c["h_last"].T @ dy, "b4": np.array([dy.sum()])}
    dA = np.outer(dy, P["w4"])
    for l in (2, 1, 0):
        dz = dA * gelu_grad(c["z"][l])
        W = ("W1", "W2", "W3")[l]
        g[("b1", "b2", "b3")[l]] = dz.sum(axis=0)
        gw = r(dz).T @ c["a"][l]
        if l == 0:
            gw[:, IN:] = 0.0
        g[W] = gw
        dA = r(dz) @ r(P[W])
    return np.concatenate([g[name].ravel() for name, _ in SHAPES]), loss
