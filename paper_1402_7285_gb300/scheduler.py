"""Learned scheduling of right-hand-side columns (host logic over GPU kernels).

Columns of the local-subspace solver converge after very different numbers of
iterations (subspace radius, vacancies, surfaces).  The scheduler predicts each
column's outer iterations to tolerance from its descriptors (tb_descriptors)
with the MLP (mlp_train / mlp_predict, GPU kernels), and orders the solver's
work queue longest-predicted-first, so the columns that finish last are
short ones and the tail of the run shrinks.  For the panel solver the same
prediction bins columns of similar length into the same panel.

The plain order (given order) is the fallback; the solver's results do not
depend on the order.  The paper has no learned component.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import Context, descriptors, mlp_param_count, mlp_predict, mlp_train

N_DESC = 32


@dataclass
class Predictor:
    params: np.ndarray   # float32 MLP parameters
    x_mean: np.ndarray   # descriptor normalisation
    x_std: np.ndarray
    y_mean: float        # target normalisation (log iterations)
    y_std: float

    def normalise(self, X):
        return ((np.asarray(X, np.float32) - self.x_mean) / self.x_std).astype(np.float32)


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), +1/sqrt(fan_in)) weights, zero biases (same layout as mlp_train)."""
    rng = np.random.default_rng(seed)
    a1, a2 = 1.0 / np.sqrt(32), 1.0 / np.sqrt(64)
    parts = [rng.uniform(-a1, a1, 64 * 32), np.zeros(64), rng.uniform(-a2, a2, 64 * 64), np.zeros(64),
             rng.uniform(-a2, a2, 64), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == mlp_param_count()
    return p


def train(ctx: Context, X, iters, *, epochs=60, batch=256, lr=2e-3, seed=0) -> tuple[Predictor, np.ndarray]:
    """Fit log(iterations) from descriptors on the GPU; returns the predictor and the loss history."""
    X = np.asarray(X, np.float32)
    y = np.log(np.maximum(np.asarray(iters, np.float64), 1.0))
    mu, sd = X.mean(axis=0), X.std(axis=0)
    sd = np.where(sd > 1e-12, sd, 1.0).astype(np.float32)
    pred = Predictor(init_params(seed), mu.astype(np.float32), sd, float(y.mean()), float(y.std() or 1.0))
    Xn = pred.normalise(X)
    yn = ((y - pred.y_mean) / pred.y_std).astype(np.float32)
    order = np.random.default_rng(seed).permutation(len(yn))   # one shuffle of the training set
    params, hist = mlp_train(ctx, Xn[order], yn[order], epochs=epochs, batch=batch, lr=lr, params=pred.params)
    pred.params = params
    return pred, hist


def predict(ctx: Context, pred: Predictor, X) -> np.ndarray:
    """Predicted outer iterations per column."""
    out = mlp_predict(ctx, pred.params, pred.normalise(X))
    out = out.cpu().numpy() if hasattr(out, "cpu") else np.asarray(out)
    return np.exp(out.astype(np.float64) * pred.y_std + pred.y_mean)


def longest_first(predicted) -> np.ndarray:
    """Queue order: descending predicted cost (stable)."""
    return np.argsort(-np.asarray(predicted), kind="stable").astype(np.int64)


def greedy_makespan(costs, order, workers: int) -> float:
    """Makespan of list scheduling: each idle worker takes the next column in `order`."""
    import heapq
    free = [0.0] * workers
    heapq.heapify(free)
    for c in order:
        t = heapq.heappop(free)
        heapq.heappush(free, t + float(costs[c]))
    return max(free)


def panels_by_prediction(predicted, width: int) -> np.ndarray:
    """Column order that puts columns of similar predicted length into the same panel."""
    return longest_first(predicted)


def padded_work(iters, order, width: int) -> float:
    """sum over panels of width * max(iterations) / sum of iterations (1 = no padding)."""
    it = np.asarray(iters, np.float64)[np.asarray(order)]
    total = 0.0
    for s in range(0, len(it), width):
        total += width * it[s:s + width].max()
    return total / it.sum()
