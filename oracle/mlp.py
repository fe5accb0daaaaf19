"""FP64 reference of the surrogate MLP (plain numpy, test infrastructure only).

Network: 3 inputs -> 4 hidden layers of 256 GELU units -> 1 output,
    z_1 = W_1 x + b_1,   a_l = GELU(z_l),   z_{l+1} = W_{l+1} a_l + b_{l+1},
    y = w_5 . a_4 + b_5,
loss = mean over the batch of (y - t)^2.  GELU in its tanh form (Hendrycks and
Gimpel, 2016): GELU(z) = z (1 + tanh(u)) / 2, u = sqrt(2/pi) (z + 0.044715 z^3),
the published approximation of z Phi(z) (Phi the standard normal CDF).

The surrogate is not part of the paper; it predicts sigma(E, t) curves that the
method generates.  Parameters use one flat FP32/FP64 layout shared with the
library's C ABI (see param_layout).

Parity: pinned by central finite differences of the loss (tests).
"""
from __future__ import annotations

import numpy as np

HIDDEN = 256
N_IN = 3
N_HIDDEN_LAYERS = 4


def param_layout(hidden: int = HIDDEN):
    """[(name, shape)] in flat order: W1 [H][3], b1, W2 [H][H], b2, W3, b3, W4, b4,
    W5 [1][H], b5 [1]."""
    out = [("W1", (hidden, N_IN)), ("b1", (hidden,))]
    for l in range(2, N_HIDDEN_LAYERS + 1):
        out += [(f"W{l}", (hidden, hidden)), (f"b{l}", (hidden,))]
    out += [("W5", (1, hidden)), ("b5", (1,))]
    return out


def n_params(hidden: int = HIDDEN) -> int:
    return int(sum(np.prod(s) for _, s in param_layout(hidden)))


def unpack(flat: np.ndarray, hidden: int = HIDDEN) -> dict:
    p, k = {}, 0
    for name, shape in param_layout(hidden):
        size = int(np.prod(shape))
        p[name] = np.asarray(flat[k:k + size], dtype=np.float64).reshape(shape)
        k += size
    return p


def pack(p: dict, hidden: int = HIDDEN) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_layout(hidden)])


def init_params(seed: int, hidden: int = HIDDEN) -> np.ndarray:
    """Uniform +-1/sqrt(fan_in) weights, zero biases (FP32 values in an FP64 array)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in param_layout(hidden):
        if name.startswith("W"):
            bound = 1.0 / np.sqrt(shape[1])
            p[name] = rng.uniform(-bound, bound, size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p, hidden).astype(np.float32).astype(np.float64)


GELU_K = np.sqrt(2.0 / np.pi)
GELU_C = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_K * (z + GELU_C * z ** 3)))


def gelu_grad(z):
    """d GELU / dz of the tanh form."""
    t = np.tanh(GELU_K * (z + GELU_C * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_K * (1.0 + 3.0 * GELU_C * z * z)


def forward(flat, x, hidden: int = HIDDEN, keep: bool = False):
    """y [B] for inputs x [B][3]; with keep, also the pre-activations and activations."""
    p = unpack(flat, hidden)
    a = np.asarray(x, dtype=np.float64)
    zs, acts = [], [a]
    for l in range(1, N_HIDDEN_LAYERS + 1):
        z = a @ p[f"W{l}"].T + p[f"b{l}"]
        a = gelu(z)
        zs.append(z)
        acts.append(a)
    y = a @ p["W5"][0] + p["b5"][0]
    return (y, zs, acts) if keep else y


def loss(flat, x, t, hidden: int = HIDDEN) -> float:
    y = forward(flat, x, hidden)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradients(flat, x, t, hidden: int = HIDDEN):
    """(loss, flat gradient) by reverse-mode differentiation of the network above."""
    p = unpack(flat, hidden)
    y, zs, acts = forward(flat, x, hidden, keep=True)
    b = len(y)
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / b
    g = {"W5": (dy @ acts[-1])[None, :], "b5": np.array([dy.sum()])}
    da = np.outer(dy, p["W5"][0])
    for l in range(N_HIDDEN_LAYERS, 0, -1):
        dz = da * gelu_grad(zs[l - 1])
        g[f"W{l}"] = dz.T @ acts[l - 1]
        g[f"b{l}"] = dz.sum(axis=0)
        da = dz @ p[f"W{l}"]
    return float(np.mean((y - t) ** 2)), pack(g, hidden)


def adam_step(flat, grad, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; returns new (flat, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
