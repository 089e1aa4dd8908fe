"""Pins of the FP64 recurrent-MLP reference (oracle/mlp.py)."""
import math

import numpy as np

from oracle import mlp


def small_problem(seed=0, B=3, T=4):
    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed)
    theta += 0.05 * rng.standard_normal(theta.shape) * (theta != 0)  # keep pads at zero
    U = rng.standard_normal((B, T, mlp.N_IN))
    Y = rng.standard_normal((B, T, mlp.N_OUT))
    return theta, U, Y


def test_gelu_closed_forms():
    x = np.linspace(-6, 6, 101)
    g = mlp.gelu(x)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # gelu(x) - gelu(-x) = x  (because Phi(x) + Phi(-x) = 1)
    assert np.abs(g - mlp.gelu(-x) - x).max() < 1e-14
    # large |x|: identity / zero
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12 and abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(x)).max() < 1e-8


def test_gpu_gelu_approximation_bounds():
    # The fused GPU kernels evaluate GELU through the tanh approximation of
    # Hendrycks & Gimpel (2016) in logistic form, x / (1 + exp(-2u)), u =
    # sqrt(2/pi) (x + 0.044715 x^3), and its derivative s + x s (1 - s) 2 u'.
    # The bounds stated for it hold against the exact GELU of the oracle.
    x = np.linspace(-12.0, 12.0, 480001)
    u = math.sqrt(2.0 / math.pi) * (x + 0.044715 * x ** 3)
    s = 1.0 / (1.0 + np.exp(-2.0 * u))
    g = x * s
    dg = s + x * s * (1.0 - s) * 2.0 * math.sqrt(2.0 / math.pi) * (1.0 + 3.0 * 0.044715 * x ** 2)
    err, derr = np.abs(g - mlp.gelu(x)), np.abs(dg - mlp.gelu_grad(x))
    assert err.max() < 4.8e-4 and 2.6 < x[err.argmax()] < 2.8
    assert derr.max() < 8.8e-4
    # at the largest deviation it is a sixteenth of the BF16 rounding (half an
    # ulp of 8 significant bits) of the value there
    i = err.argmax()
    assert err[i] < (abs(g[i]) * 2.0 ** -8) / 16.0
    # the logistic form stays finite, and non-positive below zero, out to the
    # range ends (the exponential overflows to a zero step, not to a NaN)
    assert np.all(np.isfinite(g)) and np.all(g[x < 0.0] <= 0.0)


def test_param_layout_and_padding():
    theta = mlp.init_params(1)
    assert theta.size == mlp.N_PARAMS == 144 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 144 + 144
    p = mlp.unpack(theta)
    assert np.all(p["W1"][mlp.N_IN + mlp.N_H:] == 0) and np.all(p["W4"][:, mlp.N_OUT + mlp.N_H:] == 0)
    assert np.array_equal(mlp.pack(p), theta)


def test_recurrence_is_causal_and_stateful():
    theta, U, Y = small_problem(2, B=2, T=5)
    S, _ = mlp.forward(theta, U)
    U2 = U.copy()
    U2[:, 3, :] += 1.0
    S2, _ = mlp.forward(theta, U2)
    assert np.array_equal(S[:, :3], S2[:, :3])        # the past does not see the future
    assert not np.allclose(S[:, 4], S2[:, 4])          # the hidden state carries the change forward
    # batch rows are independent
    S3, _ = mlp.forward(theta, U[:1])
    assert np.abs(S3 - S[:1]).max() < 1e-15


def test_gradient_matches_finite_differences():
    theta, U, Y = small_problem(3)
    L, g = mlp.loss_and_grad(theta, U, Y)
    assert abs(L - mlp.loss(theta, U, Y)) < 1e-15
    rng = np.random.default_rng(4)
    # every parameter block, a few coordinates each, central differences
    k = 0
    idx = []
    for name, shp in mlp.SHAPES:
        n = int(np.prod(shp))
        idx += list(k + rng.choice(n, 4, replace=False))
        k += n
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, U, Y) - mlp.loss(tm, U, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)), (i, fd, g[i])
    # directional derivative along a random direction (all parameters at once)
    d = rng.standard_normal(theta.shape)
    fd = (mlp.loss(theta + h * d, U, Y) - mlp.loss(theta - h * d, U, Y)) / (2 * h)
    assert abs(fd - g @ d) <= 1e-6 * abs(fd)


def test_adamw_closed_form_first_steps():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.2, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, wd, eps = 1e-2, 0.01, 1e-8
    t1, m, v = mlp.adamw(theta, g, m, v, 1, lr, wd=wd, eps=eps)
    # first bias-corrected step: m_hat = g, v_hat = g^2 -> lr * g / (|g| + eps), plus decay
    ref = theta - lr * (g / (np.abs(g) + eps) + wd * theta)
    assert np.abs(t1 - ref).max() < 1e-15
    # a constant gradient keeps m_hat = g, v_hat = g^2 at every step
    t2, m2, v2 = mlp.adamw(t1, g, m, v, 2, lr, wd=wd, eps=eps)
    ref2 = t1 - lr * (g / (np.abs(g) + eps) + wd * t1)
    assert np.abs(t2 - ref2).max() < 1e-15


def test_descent_on_a_fitting_problem():
    # a few hundred AdamW steps drive the loss well down on a small smooth target
    rng = np.random.default_rng(5)
    B, T = 16, 6
    U = rng.standard_normal((B, T, mlp.N_IN)) * 0.5
    Y = np.cumsum(U[:, :, :mlp.N_OUT], axis=1) * 0.3
    theta = mlp.init_params(6)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0 = mlp.loss(theta, U, Y)
    for s in range(1, 151):
        L, g = mlp.loss_and_grad(theta, U, Y)
        theta, m, v = mlp.adamw(theta, g, m, v, s, 3e-3)
    assert mlp.loss(theta, U, Y) < 0.2 * L0
    assert math.isfinite(L)


def test_features_closed_forms():
    # pure rotation: no strain; identical F: no increment; uniaxial stretch: E_xx = (l^2 - 1)/2
    th = 0.4
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    u = mlp.features(R, R)
    assert np.abs(u).max() < 1e-15
    lam = 1.2
    u = mlp.features(np.eye(3), np.diag([lam, 1.0, 1.0]))
    assert abs(u[0, 9] - 0.5 * (lam * lam - 1)) < 1e-15 and np.abs(u[0, 10:]).max() == 0.0
    assert abs(u[0, 0] - (lam - 1)) < 1e-15
    # simple shear F = I + g e_x e_y: E_xy = g/2, E_yy = g^2/2
    g = 0.1
    F = np.eye(3)
    F[0, 1] = g
    u = mlp.features(np.eye(3), F)
    assert abs(u[0, 12] - g / 2) < 1e-15 and abs(u[0, 10] - g * g / 2) < 1e-15
