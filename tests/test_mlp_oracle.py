"""Pins of the FP64 surrogate-network reference (CPU): its analytic gradient
equals central finite differences of its own forward pass, GELU matches its
closed-form values, and the BF16 rounding helper rounds to nearest even."""
import numpy as np

from oracle import mlp


def test_gelu_closed_forms():
    assert mlp.gelu(0.0) == 0.0 and abs(mlp.gelu_grad(0.0) - 0.5) < 1e-15
    assert abs(mlp.gelu(10.0) - 10.0) < 1e-12 and abs(mlp.gelu(-10.0)) < 1e-12
    z = np.linspace(-3, 3, 13)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), rtol=1e-7)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, -2.5, 3.0e-5], dtype=np.float32)
    r = mlp.to_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0  # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa
    assert r[3] == 1.0  # below halfway rounds down
    assert r[2] == 1.0 + 2 ** -7  # above halfway rounds up
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-5) / 3.0e-5 < 2 ** -8


def test_gradient_equals_finite_differences():
    rng = np.random.default_rng(0)
    n = sum(int(np.prod(s)) for _, s in mlp.SHAPES)
    p = rng.normal(0, 0.1, n)
    X = rng.uniform(0, 1, (6, mlp.IN))
    t = rng.normal(0, 1, 6)
    g, _ = mlp.gradients(p, X, t, bf16=False)
    idx = np.concatenate([rng.choice(n - 1, 40, replace=False), [n - 1]])
    h = 1e-6
    for i in idx:
        if i < mlp.H * mlp.IP and (i % mlp.IP) >= mlp.IN:
            assert g[i] == 0.0  # padding columns of W1 carry no gradient
            continue
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp = np.mean((mlp.forward(pp, X, False)[0] - t) ** 2)
        lm = np.mean((mlp.forward(pm, X, False)[0] - t) ** 2)
        assert abs(g[i] - (lp - lm) / (2 * h)) <= 1e-6 * max(1.0, abs(g[i])), i
