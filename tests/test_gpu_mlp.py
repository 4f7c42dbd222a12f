"""Tensor-core surrogate network against its FP64 reference (GPU)."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_08123_b300 import _build
    _build.build()
    return torch


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (128, 48, 48), (256, 256, 96), (384, 112, 512), (128, 256, 256),
                                   (256, 256, 4096), (128, 80, 208)])
def test_tcgen05_gemm_matches_exact_product(cuda, M, N, K):
    torch = cuda
    from paper_2303_08123_b300.surrogate import gemm_bf16
    rng = np.random.default_rng(M + N + K)
    A = mlp.to_bf16(rng.normal(0, 1, (M, K)))
    B = mlp.to_bf16(rng.normal(0, 1, (N, K)))
    At = torch.tensor(A, dtype=torch.float32).to(torch.bfloat16).cuda()
    Bt = torch.tensor(B, dtype=torch.float32).to(torch.bfloat16).cuda()
    C = gemm_bf16(At, Bt).cpu().numpy().astype(np.float64)
    want = A @ B.T  # exact in FP64 for BF16 inputs of this size
    err = np.abs(C - want) / (np.abs(A) @ np.abs(B).T + 1e-30)
    assert err.max() < 1e-5, err.max()


def _data(rng, B):
    X = rng.uniform(0, 1, (B, mlp.IN)).astype(np.float32)
    t = (X[:, 0::3].sum(axis=1) - X[:, 1::3].sum(axis=1) + 0.3 * np.sin(6 * X[:, 2])).astype(np.float32)
    return X, t


def test_forward_and_gradients_match_reference(cuda):
    from paper_2303_08123_b300.surrogate import Surrogate
    rng = np.random.default_rng(3)
    net = Surrogate(batch_max=256, seed=11)
    p = net.get_params().astype(np.float64)
    X, t = _data(rng, 256)
    y = net.forward(X).cpu().numpy()
    y_ref, _ = mlp.forward(p, X.astype(np.float64), bf16=True)
    np.testing.assert_allclose(y, y_ref, rtol=2e-3, atol=2e-3 * np.abs(y_ref).max())
    g, loss = net.gradients(X, t)
    g_ref, loss_ref = mlp.gradients(p, X.astype(np.float64), t.astype(np.float64), bf16=True)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    for name, shp in mlp.SHAPES:  # every parameter block, relative to its own scale
        o = sum(int(np.prod(s)) for n, s in mlp.SHAPES[:[n for n, _ in mlp.SHAPES].index(name)])
        n = int(np.prod(shp))
        a, b = g[o:o + n], g_ref[o:o + n]
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-12, name


def test_training_reduces_loss(cuda):
    from paper_2303_08123_b300.surrogate import Surrogate
    rng = np.random.default_rng(5)
    net = Surrogate(batch_max=512, seed=2)
    X, t = _data(rng, 512)
    first = net.train_step(X, t, 1e-3)
    for _ in range(300):
        last = net.train_step(X, t, 1e-3)
    assert last < 0.05 * first, (first, last)
    Xv, tv = _data(rng, 512)
    pred = net.predict(Xv)
    assert np.corrcoef(pred, tv)[0, 1] > 0.95


def test_bounded_wait_times_out_into_a_status_and_the_context_stays_usable(cuda):
    torch = cuda
    from paper_2303_08123_b300.surrogate import gemm_bf16, load_library
    lib = load_library()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.mlp_wait_probe(1000, st.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 1  # the wait ran out and said so
    A = torch.ones(128, 32, dtype=torch.bfloat16, device="cuda")
    C = gemm_bf16(A, A[:16])  # the device still works afterwards
    assert float(C[0, 0]) == 32.0
