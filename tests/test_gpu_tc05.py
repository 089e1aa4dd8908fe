"""The surrogate's tcgen05 paths (5th-generation tensor cores, FP32
accumulator in tensor memory) against the FP64 oracle and against the
mma.sync path, on ragged batch sizes:
  backend 1: one tcgen05 GEMM per layer and step;
  backend 2: the whole recurrent forward and the whole BPTT data-gradient
             chain each in one kernel per 128-row tile (weights streamed
             through shared memory, operands on chip), members side by side."""
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
        for be in (0, 1, 2):
            S.sur_set_backend(s, be)
            o = torch.zeros((1, B, T, 6), dtype=torch.float32, device="cuda")
            S.sur_predict(s, dU, o)
            assert S.sur_sync(s) == 0
            out[be] = o[0].cpu().numpy()
    finally:
        S.sur_destroy(s)
    ref, _ = mlp.forward(bf16_weights(theta.astype(np.float64)), bf16(U))
    scale = np.abs(ref).max()
    for be in (1, 2):
        assert np.abs(out[be] - ref).max() <= 3e-2 * scale, be
        assert np.abs(out[be] - out[0]).max() <= 2e-2 * scale, be


@pytest.mark.parametrize("backend", [1, 2])
def test_tc05_gradient_matches_oracle(torch, backend):
    B, T = 96, 6
    theta, U, Y = problem(12, B, T)
    s = S.sur_create(1, B, T, 0)
    try:
        S.sur_set_params(s, 0, theta)
        S.sur_set_backend(s, backend)
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


def test_fused_forward_members_and_long_sequence(torch):
    # three members in one launch, two row tiles with a ragged tail, 40 steps of recurrence
    B, T, K = 150, 40, 3
    thetas = [problem(20 + k, B, T)[0] for k in range(K)]
    U = problem(30, B, T)[1]
    s = S.sur_create(K, B, T, 0)
    try:
        for k in range(K):
            S.sur_set_params(s, k, thetas[k])
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        out = {}
        for be in (0, 2):
            S.sur_set_backend(s, be)
            o = torch.zeros((K, B, T, 6), dtype=torch.float32, device="cuda")
            S.sur_predict(s, dU, o)
            assert S.sur_sync(s) == 0
            out[be] = o.cpu().numpy()
    finally:
        S.sur_destroy(s)
    for k in range(K):
        ref, _ = mlp.forward(bf16_weights(thetas[k].astype(np.float64)), bf16(U))
        scale = np.abs(ref).max()
        assert np.abs(out[2][k] - ref).max() <= 1e-1 * scale, k
        assert np.abs(out[2][k] - out[0][k]).max() <= 5e-2 * scale, k


def test_fused_step_carries_state_like_the_layerwise_step(torch):
    # sur_step: one increment per call, FP32 state in and out, ensemble mean and spread
    n, K, steps = 45, 4, 6
    thetas = [problem(40 + k, n, 1)[0] for k in range(K)]
    rng = np.random.default_rng(41)
    us = rng.standard_normal((steps, n, 15)).astype(np.float32)
    res = {}
    for be in (0, 2):
        s = S.sur_create(K, n, 1, 0)
        try:
            for k in range(K):
                S.sur_set_params(s, k, thetas[k])
            S.sur_set_backend(s, be)
            h = torch.zeros((K, n, 128), dtype=torch.float32, device="cuda")
            m = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
            sp = torch.zeros(n, dtype=torch.float32, device="cuda")
            means, spreads = [], []
            for t in range(steps):
                S.sur_step(s, torch.tensor(us[t], device="cuda"), h, 0.05, m, sp)
                means.append(m.cpu().numpy().copy())
                spreads.append(sp.cpu().numpy().copy())
            assert S.sur_sync(s) == 0
            res[be] = (np.array(means), np.array(spreads), h.cpu().numpy())
        finally:
            S.sur_destroy(s)
    # the oracle's recurrence over the same increments, member by member
    U = np.transpose(us, (1, 0, 2)).astype(np.float64)
    ref = np.array([mlp.forward(bf16_weights(th.astype(np.float64)), bf16(U))[0] for th in thetas])
    ref_mean = ref.mean(0).transpose(1, 0, 2)
    scale = np.abs(ref_mean).max()
    assert np.abs(res[2][0] - ref_mean).max() <= 5e-2 * scale
    assert np.abs(res[2][0] - res[0][0]).max() <= 5e-2 * scale
    assert np.abs(res[2][2] - res[0][2]).max() <= 5e-2
    assert np.all(np.isfinite(res[2][1])) and np.abs(res[2][1] - res[0][1]).max() <= 0.1 * max(res[0][1].max(), 1e-3)


def test_member_batched_training_step_matches_oracle(torch):
    # sur_train_step on the default engine: the fused forward and the fused BPTT
    # kernel over three members at once, two row tiles with a ragged tail, 12
    # steps.  Each member's loss against the oracle, and its first AdamW update,
    # which for lr >> eps moves every parameter by about -lr sign(gradient)
    # (weight decay off), against the signs of the oracle gradient.
    B, T, K, lr = 150, 12, 3, 1e-3
    thetas = [problem(70 + k, B, T)[0] for k in range(K)]
    _, U, Y = problem(80, B, T)
    s = S.sur_create(K, B, T, 0)
    try:
        for k in range(K):
            S.sur_set_params(s, k, thetas[k])
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
        loss = S.sur_train_step(s, dU, dY, lr, wd=0.0, n_members=K)
        assert S.sur_sync(s) == 0
        after = [S.sur_get_params(s, k) for k in range(K)]
    finally:
        S.sur_destroy(s)
    for k in range(K):
        Lr, gr = mlp.loss_and_grad(bf16_weights(thetas[k].astype(np.float64)), bf16(U), Y)
        assert abs(loss[k] - Lr) <= 2e-2 * Lr, (k, loss[k], Lr)
        step = after[k].astype(np.float64) - thetas[k].astype(np.float64)
        big = np.abs(gr) > 1e-2 * np.abs(gr).max()
        agree = np.mean(np.sign(step[big]) == -np.sign(gr[big]))
        assert agree > 0.99, (k, agree)
        assert np.abs(step[big]).max() <= 1.01 * lr


def test_profile_step_times_the_phases_and_changes_no_parameter(torch):
    B, T, K = 150, 8, 2
    thetas = [problem(90 + k, B, T)[0] for k in range(K)]
    _, U, Y = problem(91, B, T)
    s = S.sur_create(K, B, T, 0)
    try:
        for k in range(K):
            S.sur_set_params(s, k, thetas[k])
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
        ph = S.sur_profile_step(s, dU, dY)
        assert S.sur_sync(s) == 0
        assert set(ph) == {"forward_tape", "backward", "weight_grad"} and min(ph.values()) > 0.0
        for k in range(K):
            assert np.array_equal(S.sur_get_params(s, k), thetas[k])
    finally:
        S.sur_destroy(s)
