"""Float64 reference of the learned k-th-distance regressor -- TEST INFRASTRUCTURE ONLY.

The regressor (a design choice on top of the paper's nearest traversal, which
it only seeds with an initial bound) maps a query to an estimate of log d_k,
the distance to its k-th nearest primitive:

    x  = (q - L) / (H - L)                 (scene-box normalisation, 0 on a flat axis)
    h1 = relu(W1 x + b1)                   W1: 64 x 3
    h2 = relu(W2 h1 + b2)                  W2: 64 x 64
    y  = w3 . h2 + b3                      w3: 64
    loss = mean over the batch of (y - t)^2,  t = log(max(d_k, 1e-30))

Backward is the textbook chain rule for this composition; Adam follows Kingma
& Ba (2015), Algorithm 1, with bias-corrected moments.  Parameters are kept in
one flat vector in the order W1, b1, W2, b2, w3, b3 (row-major matrices).
"""
from __future__ import annotations

import numpy as np

H = 64
SIZES = (("W1", (H, 3)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)  # 4481


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        sz = int(np.prod(shape))
        out[name] = theta[o:o + sz].reshape(shape)
        o += sz
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SIZES])


def normalise(q: np.ndarray, scene: np.ndarray) -> np.ndarray:
    q = np.asarray(q, np.float64)
    lo = np.asarray(scene[:3], np.float64)
    hi = np.asarray(scene[3:], np.float64)
    ext = hi - lo
    safe = np.where(ext > 0, ext, 1.0)
    return np.where(ext > 0, (q - lo) / safe, 0.0)


def label(dk2: np.ndarray) -> np.ndarray:
    """t = log(max(d_k, 1e-30)) from the k-th squared distance."""
    d = np.sqrt(np.asarray(dk2, np.float64))
    return np.log(np.maximum(d, 1e-30))


def forward(theta: np.ndarray, x: np.ndarray):
    p = unpack(np.asarray(theta, np.float64))
    x = np.asarray(x, np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss(theta: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(theta, x)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def backward(theta: np.ndarray, x: np.ndarray, t: np.ndarray):
    """(loss, gradient of the mean squared error w.r.t. the flat parameters)."""
    p = unpack(np.asarray(theta, np.float64))
    y, (x, z1, h1, z2, h2) = forward(theta, x)
    nb = x.shape[0]
    r = y - np.asarray(t, np.float64)
    dy = 2.0 * r / nb
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean(r * r)), pack(g)


class Adam:
    """Adam with bias correction; state in float64."""

    def __init__(self, n: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta: np.ndarray, grad: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        mhat = self.m / (1.0 - self.b1 ** self.t)
        vhat = self.v / (1.0 - self.b2 ** self.t)
        return theta - self.lr * mhat / (np.sqrt(vhat) + self.eps)


def he_init(seed_rng: np.random.Generator) -> np.ndarray:
    """He-normal weights, zero biases, output bias 0."""
    p = {
        "W1": seed_rng.standard_normal((H, 3)) * np.sqrt(2.0 / 3.0),
        "b1": np.zeros(H),
        "W2": seed_rng.standard_normal((H, H)) * np.sqrt(2.0 / H),
        "b2": np.zeros(H),
        "w3": seed_rng.standard_normal(H) * np.sqrt(1.0 / H),
        "b3": np.zeros(1),
    }
    return pack(p)
