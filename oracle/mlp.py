"""FP64 multilayer perceptron for the iteration-count predictor (oracle side).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

The paper has no learned component; this predictor is part of the project's
scheduler (per-column iterations-to-tolerance, used to order right-hand sides
so that columns of similar length share a panel).  Architecture:
    h1 = tanh(W1 x + b1)      W1: [64, 32]
    h2 = tanh(W2 h1 + b2)     W2: [64, 64]
    y  = w3 . h2 + b3         w3: [64]
Loss: mean squared error over a batch, L = mean_i (y_i - t_i)^2.
Optimizer: Adam (Kingma & Ba, 2015) with bias correction:
    m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
    p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
Forward and backward are written out layer by layer with numpy matmuls.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

D_IN, D_H = 32, 64
PARAM_NAMES = ("W1", "b1", "W2", "b2", "w3", "b3")


def init_params(seed: int) -> dict:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    a1, a2 = 1.0 / np.sqrt(D_IN), 1.0 / np.sqrt(D_H)
    return {
        "W1": rng.uniform(-a1, a1, (D_H, D_IN)), "b1": np.zeros(D_H),
        "W2": rng.uniform(-a2, a2, (D_H, D_H)), "b2": np.zeros(D_H),
        "w3": rng.uniform(-a2, a2, D_H), "b3": np.zeros(1),
    }


def forward(p: dict, X: np.ndarray):
    """X [n, 32] -> (y [n], cache)."""
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, h1, h2)


def loss(p: dict, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(p, X)
    return float(np.mean((y - t) ** 2))


def backward(p: dict, X: np.ndarray, t: np.ndarray) -> dict:
    """Gradients of the mean squared error with respect to every parameter."""
    y, (X, h1, h2) = forward(p, X)
    n = X.shape[0]
    dy = 2.0 * (y - t) / n                     # dL/dy
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dh2 = np.outer(dy, p["w3"])                # [n, 64]
    dz2 = dh2 * (1.0 - h2 * h2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (1.0 - h1 * h1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return g


@dataclass
class Adam:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: dict = field(default_factory=dict)
    v: dict = field(default_factory=dict)

    def step(self, p: dict, g: dict) -> None:
        self.t += 1
        for k in PARAM_NAMES:
            if k not in self.m:
                self.m[k] = np.zeros_like(p[k])
                self.v[k] = np.zeros_like(p[k])
            self.m[k] = self.beta1 * self.m[k] + (1.0 - self.beta1) * g[k]
            self.v[k] = self.beta2 * self.v[k] + (1.0 - self.beta2) * g[k] * g[k]
            mh = self.m[k] / (1.0 - self.beta1 ** self.t)
            vh = self.v[k] / (1.0 - self.beta2 ** self.t)
            p[k] = p[k] - self.lr * mh / (np.sqrt(vh) + self.eps)


def train(p: dict, X: np.ndarray, t: np.ndarray, epochs: int, batch: int, lr: float, seed: int) -> list:
    """Minibatch Adam; the batch order of each epoch is a seeded permutation."""
    opt = Adam(lr=lr)
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        perm = rng.permutation(X.shape[0])
        for s in range(0, X.shape[0], batch):
            idx = perm[s:s + batch]
            opt.step(p, backward(p, X[idx], t[idx]))
        hist.append(loss(p, X, t))
    return hist
