"""The float64 selector network of the oracle, pinned by finite differences,
closed forms and a separable toy problem."""
import math

import numpy as np

from oracle import mlp as M


def _batch(seed, B=16):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, M.IN))
    y = rng.integers(0, M.OUT, B)
    mask = rng.random((B, M.OUT)) < 0.7
    mask[np.arange(B), y] = True
    return X, y, mask


def test_layout():
    assert M.NPARAMS == 64 * 32 + 64 + 64 * 64 + 64 + 12 * 64 + 12 == 7052
    p = np.arange(M.NPARAMS, dtype=np.float64)
    assert np.array_equal(M.pack(M.unpack(p)), p)
    assert M.unpack(p)["W1"][1, 0] == 32 and M.unpack(p)["b3"][0] == 7040


def test_gradient_matches_central_differences():
    X, y, mask = _batch(1)
    p = M.he_init(3) + 0.01 * np.random.default_rng(4).normal(size=M.NPARAMS)
    loss, g = M.loss_grad(p, X, y, mask)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(M.NPARAMS, 300, replace=False), [0, 2047, 2048, 7039, 7051]])
    eps = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += eps
        lp, _ = M.loss_grad(q, X, y, mask)
        q[i] -= 2 * eps
        lm, _ = M.loss_grad(q, X, y, mask)
        num = (lp - lm) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 + 1e-4 * abs(num), (i, num, g[i])


def test_zero_weights_give_uniform_softmax():
    X, y, mask = _batch(2)
    loss, g = M.loss_grad(np.zeros(M.NPARAMS), X, y, mask)
    k = mask.sum(1)
    assert math.isclose(loss, float(np.log(k).mean()), rel_tol=1e-12)
    # only b3 has a gradient: mean over the batch of (1/k on allowed classes) - onehot(y)
    gb3 = M.unpack(g)["b3"]
    expect = (mask / k[:, None]).mean(0)
    expect -= np.bincount(y, minlength=M.OUT) / len(y)
    assert np.allclose(gb3, expect, atol=1e-15)
    assert np.all(M.unpack(g)["W1"] == 0) and np.all(M.unpack(g)["W3"] == 0)


def test_adam_first_step_moves_by_lr_times_sign():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = M.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p[:3], -0.01 * np.sign(g[:3]), rtol=1e-5) and p[3] == 0


def test_masked_classes_never_predicted_and_separable_toy_learned():
    rng = np.random.default_rng(7)
    centers = rng.normal(size=(M.OUT, M.IN)) * 3
    y = rng.integers(0, M.OUT, 600)
    X = centers[y] + 0.3 * rng.normal(size=(600, M.IN))
    mask = np.ones((600, M.OUT), bool)
    p = M.train(X, y, mask, epochs=60, batch=64, lr=3e-3, seed=1)
    assert (M.predict(p, X, mask) == y).mean() == 1.0
    mask2 = mask.copy()
    mask2[:, 0] = False
    assert not np.any(M.predict(p, X, mask2) == 0)
