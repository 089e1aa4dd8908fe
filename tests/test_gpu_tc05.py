"""The surrogate's tcgen05 GEMM path (5th-generation tensor cores, FP32
accumulator in tensor memory) against the FP64 oracle and against the
mma.sync path, on ragged batch sizes."""
import numpy as np
import pytest

from oracle import mlp
from paper_1902_09171_gb300 import surrogate as S
from test_gpu_surrogate import bf16, bf16_weights, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    from paper_1902_09171_gb300 import build
    build.build()
    return t


@pytest.mark.parametrize("B", [200, 37])
def test_tc05_forward_matches_oracle_and_mma(torch, B):
    T = 5
    theta, U, _ = problem(11, B, T)
    s = S.sur_create(1, B, T, 0)
    try:
        S.sur_set_params(s, 0, theta)
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        out = {}
        for be in (0, 1):
            S.sur_set_backend(s, be)
            o = torch.zeros((1, B, T, 6), dtype=torch.float32, device="cuda")
            S.sur_predict(s, dU, o)
            assert S.sur_sync(s) == 0
            out[be] = o[0].cpu().numpy()
    finally:
        S.sur_destroy(s)
    ref, _ = mlp.forward(bf16_weights(theta.astype(np.float64)), bf16(U))
    scale = np.abs(ref).max()
    assert np.abs(out[1] - ref).max() <= 3e-2 * scale
    assert np.abs(out[1] - out[0]).max() <= 2e-2 * scale


def test_tc05_gradient_matches_oracle(torch):
    B, T = 96, 6
    theta, U, Y = problem(12, B, T)
    s = S.sur_create(1, B, T, 0)
    try:
        S.sur_set_params(s, 0, theta)
        S.sur_set_backend(s, 1)
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
        L, g = S.sur_loss_grad(s, 0, dU, dY)
        assert S.sur_sync(s) == 0
    finally:
        S.sur_destroy(s)
    Lr, gr = mlp.loss_and_grad(bf16_weights(theta.astype(np.float64)), bf16(U), Y)
    rel = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    cos = g @ gr / (np.linalg.norm(g) * np.linalg.norm(gr))
    assert abs(L - Lr) <= 2e-2 * Lr and rel <= 5e-2 and cos > 0.999, (rel, cos)
