"""Pins of the surrogate network's CPU oracle (oracle/mlp.py).

The network, loss and optimiser follow the paper's Table "para-setting"
(Sec. 3.3), which the authors ran in scikit-learn; scikit-learn (when
importable) is an independent implementation of the same definitions.
"""
import numpy as np
import pytest

from oracle import mlp as M


def _data(n=300, nin=5, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, nin))
    y = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.2 * X[:, 3] + 0.05 * rng.normal(size=n)
    return X, y


def test_backprop_gradients_match_central_differences():
    X, y = _data(40, 4)
    sizes = [4, 7, 5, 1]
    rng = np.random.default_rng(1)
    params = M.glorot_init(sizes, rng.random(M.n_params(sizes)))
    loss, grads = M.loss_and_grads(params, X, y, alpha=1e-2)
    h = 1e-6
    for p, g in zip(params, grads):
        flat, gflat = p.reshape(-1), g.reshape(-1)
        for k in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[k]
            flat[k] = old + h
            lp, _ = M.loss_and_grads(params, X, y, alpha=1e-2)
            flat[k] = old - h
            lm, _ = M.loss_and_grads(params, X, y, alpha=1e-2)
            flat[k] = old
            assert abs((lp - lm) / (2 * h) - gflat[k]) <= 1e-7 * max(1.0, abs(gflat[k]))


def test_adam_first_step_has_the_closed_form_size():
    # after one step from zero moments every parameter moves by lr * g / (|g| + eps) (bias-corrected)
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -1e-3, 2.0])]
    opt = M.Adam(p, lr=0.1, beta1=0.95, beta2=0.9, eps=1e-9)
    before = p[0].copy()
    opt.step(p, g)
    lr_t = 0.1 * np.sqrt(1 - 0.9) / (1 - 0.95)
    expect = before - lr_t * (0.05 * g[0]) / (np.sqrt(0.1 * g[0] ** 2) + 1e-9)
    np.testing.assert_allclose(p[0], expect, rtol=1e-15)
    np.testing.assert_allclose(before - p[0], 0.1 * np.sign(g[0]), rtol=1e-5)


def test_one_epoch_matches_scikit_learn():
    sk = pytest.importorskip("sklearn.neural_network")
    X, y = _data(450, 5)
    sizes = [5, 16, 8, 1]
    rng = np.random.default_rng(2)
    params = M.glorot_init(sizes, rng.random(M.n_params(sizes)))
    h = M.HYPER
    reg = sk.MLPRegressor(hidden_layer_sizes=tuple(sizes[1:-1]), activation="relu", solver="adam",
                          alpha=h["alpha"], batch_size=h["batch"], learning_rate_init=h["lr"], beta_1=h["beta1"],
                          beta_2=h["beta2"], epsilon=h["eps"], shuffle=False, max_iter=1)
    reg._random_state = np.random.RandomState(0)
    reg._initialize(y.reshape(-1, 1), [5] + sizes[1:-1] + [1], np.float64)
    reg.coefs_ = [p.copy() for p in params[0::2]]
    reg.intercepts_ = [p.copy() for p in params[1::2]]
    for _ in range(3):
        reg.partial_fit(X, y)
    ours = [p.copy() for p in params]
    opt = M.Adam(ours, h["lr"], h["beta1"], h["beta2"], h["eps"])
    # three epochs in order, continuing one optimiser (partial_fit keeps its Adam state)
    for _ in range(3):
        for s in range(0, 450, h["batch"]):
            idx = np.arange(s, min(s + h["batch"], 450))
            _, grads = M.loss_and_grads(ours, X[idx], y[idx], h["alpha"])
            opt.step(ours, grads)
    for a, b in zip(ours[0::2], reg.coefs_):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)
    for a, b in zip(ours[1::2], reg.intercepts_):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_r2_matches_scikit_learn_and_training_fits():
    metrics = pytest.importorskip("sklearn.metrics")
    X, y = _data(600, 5, seed=4)
    Xs = M.standardize(X[:450], X)
    sizes = [5, 32, 16, 1]
    params = M.glorot_init(sizes, np.random.default_rng(5).random(M.n_params(sizes)))
    rng = np.random.default_rng(6)
    order = np.stack([rng.permutation(450) for _ in range(200)])
    losses = M.train(params, Xs[:450], y[:450], order)
    assert losses[-1] < 0.1 * losses[0]
    yhat = M.predict(params, Xs[450:])
    assert abs(M.r2(y[450:], yhat) - metrics.r2_score(y[450:], yhat)) < 1e-14
    assert M.r2(y[450:], yhat) > 0.6
