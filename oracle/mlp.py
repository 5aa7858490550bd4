"""CPU oracle of the autotuner's surrogate network: TEST INFRASTRUCTURE ONLY.

A plain NumPy FP64 fully connected network, written from the paper's Sec. 3.3
(Table "para-setting"; Eq. (7) for R^2) and the definitions it relies on:
  * layers: ReLU hidden layers, identity output (a regressor of run time);
  * loss per minibatch of size B: 1/2 mean((y_hat - y)^2) + alpha/(2B) sum ||W||^2
    (L2 on weights, not biases; alpha = 1e-4);
  * gradients by backpropagation: dW = (A^T delta + alpha W) / B, db = mean(delta);
  * Adam (Kingma & Ba 2015) in the authors' efficient form:
      m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
      lr_t = lr sqrt(1 - b2^t) / (1 - b1^t),  theta <- theta - lr_t m / (sqrt(v) + eps)
    with b1 = 0.95, b2 = 0.90, lr = 0.0009, eps = 1e-9 (constant rate: the
    "adaptive" schedule of the table has no meaning for Adam);
  * training: minibatches of 200 in a given order, at most 200 epochs, stop
    once the epoch loss has failed to improve by tol = 1e-6 for 10 epochs;
  * features centred and scaled (StandardScaler, Sec. 3.5);
  * R^2 = 1 - sum (y - y_hat)^2 / sum (y - mean y)^2 (Eq. (7)).
Weights are stored as the list [W_0, b_0, W_1, b_1, ...], W_l of shape
(fan_in, fan_out).
"""
from __future__ import annotations

import numpy as np

HYPER = dict(alpha=1e-4, beta1=0.95, beta2=0.90, lr=9e-4, eps=1e-9, batch=200, epochs=200, tol=1e-6,
             n_iter_no_change=10)


def glorot_init(sizes, uniform01):
    """Weights with the Glorot-uniform bound sqrt(6 / (fan_in + fan_out)), for
    weights and biases, from a supplied stream of U[0, 1) numbers (so that
    CPU and GPU start from identical parameters)."""
    params = []
    k = 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        bound = np.sqrt(6.0 / (fi + fo))
        W = (2.0 * uniform01[k:k + fi * fo].reshape(fi, fo) - 1.0) * bound
        k += fi * fo
        b = (2.0 * uniform01[k:k + fo] - 1.0) * bound
        k += fo
        params += [W, b]
    return params


def n_params(sizes) -> int:
    return sum(fi * fo + fo for fi, fo in zip(sizes[:-1], sizes[1:]))


def forward(params, X):
    """Activations of every layer (input first); ReLU hidden, identity output."""
    acts = [X]
    L = len(params) // 2
    for l in range(L):
        Z = acts[-1] @ params[2 * l] + params[2 * l + 1]
        acts.append(np.maximum(Z, 0.0) if l < L - 1 else Z)
    return acts


def predict(params, X):
    return forward(params, X)[-1][:, 0]


def loss_and_grads(params, X, y, alpha):
    B = X.shape[0]
    acts = forward(params, X)
    L = len(params) // 2
    out = acts[-1][:, 0]
    loss = 0.5 * np.mean((out - y) ** 2) + 0.5 * alpha * sum(np.sum(params[2 * l] ** 2) for l in range(L)) / B
    delta = (out - y)[:, None]
    grads = [None] * len(params)
    for l in range(L - 1, -1, -1):
        grads[2 * l] = (acts[l].T @ delta + alpha * params[2 * l]) / B
        grads[2 * l + 1] = delta.mean(axis=0)
        if l > 0:
            delta = (delta @ params[2 * l].T) * (acts[l] > 0.0)
    return loss, grads


class Adam:
    def __init__(self, params, lr, beta1, beta2, eps):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.t = 0
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]

    def step(self, params, grads):
        self.t += 1
        lr_t = self.lr * np.sqrt(1.0 - self.b2 ** self.t) / (1.0 - self.b1 ** self.t)
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.b1
            m += (1.0 - self.b1) * g
            v *= self.b2
            v += (1.0 - self.b2) * g * g
            p -= lr_t * m / (np.sqrt(v) + self.eps)


def train(params, X, y, order, hyper=None):
    """Train in place.  order: (epochs, n) sample indices per epoch; batches are
    consecutive slices of `batch` indices (the last may be shorter).
    Returns the per-epoch losses (mean over samples) actually run."""
    h = dict(HYPER, **(hyper or {}))
    opt = Adam(params, h["lr"], h["beta1"], h["beta2"], h["eps"])
    n = X.shape[0]
    losses = []
    best, bad = np.inf, 0
    for e in range(order.shape[0]):
        acc = 0.0
        for s in range(0, n, h["batch"]):
            idx = order[e, s:s + h["batch"]]
            loss, grads = loss_and_grads(params, X[idx], y[idx], h["alpha"])
            opt.step(params, grads)
            acc += loss * idx.size
        losses.append(acc / n)
        if losses[-1] > best - h["tol"]:
            bad += 1
        else:
            bad = 0
        best = min(best, losses[-1])
        if bad > h["n_iter_no_change"]:
            break
    return losses


def standardize(Xtr, X):
    mu = Xtr.mean(axis=0)
    sd = Xtr.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    return (X - mu) / sd


def r2(y, yhat):
    """Eq. (7)."""
    y = np.asarray(y, dtype=np.float64)
    return 1.0 - np.sum((y - yhat) ** 2) / np.sum((y - y.mean()) ** 2)
