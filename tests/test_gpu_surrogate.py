"""GPU-vs-oracle parity of the recurrent-MLP surrogate kernels (BF16 tensor
cores, FP32 accumulation) against the FP64 NumPy reference oracle/mlp.py.

Tolerances: the GPU rounds weights and activations to BF16 (8-bit mantissa,
relative rounding 2^-9 = 2e-3 per value); forward predictions are compared at
3e-2 of their scale, gradients at relative L2 error 5e-2 with cosine > 0.999
(gradients are taken with BF16-rounded weights and inputs on both sides).
"""
import numpy as np
import pytest

from oracle import mlp
from paper_1902_09171_gb300 import surrogate as S

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


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    x = np.asarray(a, dtype=np.float32).copy()
    u = x.view(np.uint32)
    u += ((u >> 16) & 1) + np.uint32(0x7FFF)
    u &= np.uint32(0xFFFF0000)
    return x.astype(np.float64)


def bf16_weights(theta):
    p = mlp.unpack(theta)
    for k in ("W1", "W2", "W3", "W4"):
        p[k] = bf16(p[k])
    return mlp.pack(p)


def problem(seed, B, T):
    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed)
    U = rng.standard_normal((B, T, mlp.N_IN))
    Y = 0.5 * np.cumsum(U[:, :, :mlp.N_OUT], axis=1)
    return theta.astype(np.float32), U, Y


def test_forward_matches_oracle(torch):
    B, T = 96, 7  # ragged against the 64-row tiles
    theta, U, Y = problem(1, B, T)
    s = S.sur_create(1, B, T, 0)
    try:
        S.sur_set_params(s, 0, theta)
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        out = torch.zeros((1, B, T, 6), dtype=torch.float32, device="cuda")
        S.sur_predict(s, dU, out)
        torch.cuda.synchronize()
        got = out[0].cpu().numpy()
    finally:
        S.sur_destroy(s)
    ref, _ = mlp.forward(bf16_weights(theta.astype(np.float64)), bf16(U))
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 3e-2 * scale
    assert np.abs(got - ref).mean() <= 5e-3 * scale


def test_gradient_matches_oracle(torch):
    B, T = 64, 6
    theta, U, Y = problem(2, B, T)
    s = S.sur_create(1, B, T, 0)
    try:
        S.sur_set_params(s, 0, theta)
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
        L, g = S.sur_loss_grad(s, 0, dU, dY)
    finally:
        S.sur_destroy(s)
    Lr, gr = mlp.loss_and_grad(bf16_weights(theta.astype(np.float64)), bf16(U), Y)
    assert abs(L - Lr) <= 2e-2 * Lr
    rel = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    cos = g @ gr / (np.linalg.norm(g) * np.linalg.norm(gr))
    assert rel <= 5e-2 and cos > 0.999, (rel, cos)
    # every parameter block individually
    k = 0
    for name, shp in mlp.SHAPES:
        n = int(np.prod(shp))
        gb, rb = g[k:k + n], gr[k:k + n]
        k += n
        if np.linalg.norm(rb) == 0:
            assert np.linalg.norm(gb) < 1e-6
            continue
        assert np.linalg.norm(gb - rb) / np.linalg.norm(rb) <= 8e-2, name


def test_adamw_step_matches_oracle_update(torch):
    B, T = 64, 4
    theta, U, Y = problem(3, B, T)
    s = S.sur_create(1, B, T, 0)
    try:
        S.sur_set_params(s, 0, theta)
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
        _, g = S.sur_loss_grad(s, 0, dU, dY)
        S.sur_train_step(s, dU, dY, lr=1e-3, wd=0.01)
        th1 = S.sur_get_params(s, 0)
    finally:
        S.sur_destroy(s)
    ref, _, _ = mlp.adamw(theta.astype(np.float64), g.astype(np.float64), np.zeros(theta.size), np.zeros(theta.size),
                          1, 1e-3, wd=0.01)
    # the first AdamW step moves every parameter with |g| >> eps by lr * sign(g) (+ decay)
    big = np.abs(g) > 1e-5
    assert np.abs(th1 - ref)[big].max() <= 2e-6
    assert np.abs(th1 - theta).max() <= 1.01e-3 + 1e-5 * np.abs(theta).max()


def test_training_reduces_loss(torch):
    B, T = 256, 8
    rng = np.random.default_rng(4)
    U = rng.standard_normal((B, T, mlp.N_IN)) * 0.5
    Y = 0.3 * np.cumsum(U[:, :, :mlp.N_OUT], axis=1)
    s = S.sur_create(2, B, T, 7)
    try:
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
        first = S.sur_train_step(s, dU, dY, lr=2e-3, n_members=2)
        for _ in range(300):
            last = S.sur_train_step(s, dU, dY, lr=2e-3, n_members=2, want_loss=False)
        last = S.sur_train_step(s, dU, dY, lr=2e-3, n_members=2)
    finally:
        S.sur_destroy(s)
    assert np.all(last < 0.1 * first), (first, last)


def test_step_inference_equals_sequence_prediction(torch):
    # sur_step applied T times with its recurrent state reproduces sur_predict;
    # two members with identical parameters have zero spread
    B, T = 40, 5
    theta, U, _ = problem(5, B, T)
    s = S.sur_create(2, B, T, 0)
    try:
        S.sur_set_params(s, 0, theta)
        S.sur_set_params(s, 1, theta)
        S.sur_set_scaling(s, np.full(15, 2.0), np.full(6, 3.0))
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        seq = torch.zeros((2, B, T, 6), dtype=torch.float32, device="cuda")
        S.sur_predict(s, dU, seq)
        h = torch.zeros((2, B, 128), dtype=torch.float32, device="cuda")
        mean = torch.zeros((B, 6), dtype=torch.float32, device="cuda")
        spread = torch.zeros((B,), dtype=torch.float32, device="cuda")
        steps = []
        for t in range(T):
            u_t = dU[:, t, :].contiguous()
            S.sur_step(s, u_t, h, 1e-3, mean, spread)
            torch.cuda.synchronize()
            steps.append(mean.cpu().numpy().copy())
            assert float(spread.abs().max()) == 0.0
        got = np.stack(steps, axis=1)
        ref = seq[0].cpu().numpy()
    finally:
        S.sur_destroy(s)
    # the step path keeps the state in FP32 between steps, the sequence path in BF16
    assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max()
    # scaling: outputs are the network outputs times s_scale = 3 on inputs / 2
    net, _ = mlp.forward(bf16_weights(theta.astype(np.float64)), bf16(U / 2.0))
    assert np.abs(ref - 3.0 * net).max() <= 3e-2 * np.abs(3.0 * net).max()


def test_ensemble_spread_of_different_members(torch):
    B = 32
    rng = np.random.default_rng(6)
    u = rng.standard_normal((B, 15))
    s = S.sur_create(4, B, 1, 11)
    try:
        du = torch.tensor(u, dtype=torch.float32, device="cuda")
        h = torch.zeros((4, B, 128), dtype=torch.float32, device="cuda")
        mean = torch.zeros((B, 6), dtype=torch.float32, device="cuda")
        spread = torch.zeros((B,), dtype=torch.float32, device="cuda")
        S.sur_step(s, du, h, 1e-6, mean, spread)
        seq = torch.zeros((4, B, 1, 6), dtype=torch.float32, device="cuda")
        S.sur_predict(s, du.view(B, 1, 15).contiguous(), seq)
        torch.cuda.synchronize()
        Sm = seq[:, :, 0, :].cpu().numpy()
    finally:
        S.sur_destroy(s)
    mu = Sm.mean(0)
    sd = np.sqrt(((Sm - mu) ** 2).sum(0) / 3).sum(-1)
    ref = np.sqrt((Sm.std(0, ddof=1) ** 2).sum(-1)) / np.maximum(np.linalg.norm(mu, axis=-1), 1e-6)
    assert np.abs(mean.cpu().numpy() - mu).max() <= 1e-5 * np.abs(mu).max() + 1e-6
    assert np.abs(spread.cpu().numpy() - ref).max() <= 1e-3 * ref.max()
    assert np.all(sd > 0)
