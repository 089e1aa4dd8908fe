"""FP64 NumPy reference of the recurrent-MLP stress surrogate -- TEST INFRASTRUCTURE.

Only the test suite may use this module.  It is the plain definition that the
GPU's BF16 tensor-core kernels are checked against (same architecture, FP64,
no blocking or fusion).  The paper itself has no learned component; the model
follows the surrogate specification of the hot path: a recurrent MLP that maps
the strain-increment history of a quadrature point to its stress.

Architecture (one time step t, batch rows independent):
    z_t   = [u_t (15 features), h_{t-1} (128), 0 (1 pad)]            (144)
    y_1   = z_t W1 + b1,  a_1 = gelu(y_1)                            (256)
    y_2   = a_1 W2 + b2,  a_2 = gelu(y_2)                            (256)
    y_3   = a_2 W3 + b3,  a_3 = gelu(y_3)                            (256)
    o_t   = a_3 W4 + b4                                              (144)
    s_t   = o_t[0:6]   (normalised stress)
    h_t   = tanh(o_t[6:134]);  o_t[134:144] unused (padding)
with h_0 = 0 and gelu(x) = x/2 (1 + erf(x / sqrt 2)).
Loss: mean over (batch, time, 6 components) of (s_t - target_t)^2.
Parameters are kept in one flat FP32/FP64 vector in the order
W1, b1, W2, b2, W3, b3, W4, b4 (weights row-major, K x N).
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H, N_OUT, WIDTH = 15, 128, 6, 256
K0 = 144          # padded input width  (15 + 128 + 1)
N4 = 144          # padded head width   (6 + 128 + 10)
SHAPES = [("W1", (K0, WIDTH)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("W4", (WIDTH, N4)), ("b4", (N4,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)

_erf = np.vectorize(math.erf)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def unpack(theta):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shp)
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed):
    """Seeded initialisation (uniform +-1/sqrt(fan_in) weights, zero biases); pads are zero."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = 1.0 / math.sqrt(shp[0])
            p[name] = rng.uniform(-lim, lim, size=shp)
        else:
            p[name] = np.zeros(shp)
    p["W1"][N_IN + N_H:, :] = 0.0       # padding row of the input
    p["W4"][:, N_OUT + N_H:] = 0.0      # padding columns of the head
    p["b4"][N_OUT + N_H:] = 0.0
    return pack(p)


def forward(theta, U):
    """U: (B, T, 15) features.  Returns predictions (B, T, 6) and the tape."""
    p = unpack(theta)
    B, T, _ = U.shape
    h = np.zeros((B, N_H))
    S = np.zeros((B, T, N_OUT))
    tape = []
    for t in range(T):
        z = np.concatenate([U[:, t, :], h, np.zeros((B, K0 - N_IN - N_H))], axis=1)
        y1 = z @ p["W1"] + p["b1"]
        a1 = gelu(y1)
        y2 = a1 @ p["W2"] + p["b2"]
        a2 = gelu(y2)
        y3 = a2 @ p["W3"] + p["b3"]
        a3 = gelu(y3)
        o = a3 @ p["W4"] + p["b4"]
        S[:, t, :] = o[:, :N_OUT]
        h = np.tanh(o[:, N_OUT:N_OUT + N_H])
        tape.append((z, y1, a1, y2, a2, y3, a3, o, h))
    return S, tape


def loss(theta, U, Y):
    S, _ = forward(theta, U)
    return float(np.mean((S - Y) ** 2))


def loss_and_grad(theta, U, Y):
    """Mean-squared loss and its gradient by back-propagation through time."""
    p = unpack(theta)
    S, tape = forward(theta, U)
    B, T, _ = U.shape
    scale = 2.0 / (B * T * N_OUT)
    g = {name: np.zeros(shp) for name, shp in SHAPES}
    dh = np.zeros((B, N_H))
    for t in reversed(range(T)):
        z, y1, a1, y2, a2, y3, a3, o, h = tape[t]
        do = np.zeros((B, N4))
        do[:, :N_OUT] = scale * (S[:, t, :] - Y[:, t, :])
        do[:, N_OUT:N_OUT + N_H] = dh * (1.0 - h * h)
        g["W4"] += a3.T @ do
        g["b4"] += do.sum(0)
        dy3 = (do @ p["W4"].T) * gelu_grad(y3)
        g["W3"] += a2.T @ dy3
        g["b3"] += dy3.sum(0)
        dy2 = (dy3 @ p["W3"].T) * gelu_grad(y2)
        g["W2"] += a1.T @ dy2
        g["b2"] += dy2.sum(0)
        dy1 = (dy2 @ p["W2"].T) * gelu_grad(y1)
        g["W1"] += z.T @ dy1
        g["b1"] += dy1.sum(0)
        dz = dy1 @ p["W1"].T
        dh = dz[:, N_IN:N_IN + N_H]
    return float(np.mean((S - Y) ** 2)), pack(g)


def adamw(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01):
    """One AdamW step (Loshchilov & Hutter): decoupled weight decay on every
    parameter, bias-corrected first and second moments.  `step` counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v


def features(F_prev, F):
    """Surrogate input of one increment: (F - F_prev) row-major (9) and the Green
    strain E = (F^T F - I)/2 in Voigt order xx yy zz xy xz yz (6)."""
    F_prev = np.asarray(F_prev, dtype=np.float64).reshape(-1, 3, 3)
    F = np.asarray(F, dtype=np.float64).reshape(-1, 3, 3)
    E = 0.5 * (np.einsum("nki,nkj->nij", F, F) - np.eye(3))
    v = np.stack([E[:, 0, 0], E[:, 1, 1], E[:, 2, 2], E[:, 0, 1], E[:, 0, 2], E[:, 1, 2]], axis=1)
    return np.concatenate([(F - F_prev).reshape(-1, 9), v], axis=1)
