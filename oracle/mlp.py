"""The selector network in float64 numpy -- test infrastructure.

A multilayer perceptron 32 -> 64 -> 64 -> 12 with ReLU hidden layers,
softmax cross-entropy over the classes a sample allows (the others are
masked out), mean over the batch, and the Adam update (Kingma & Ba 2015):
m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr * (m / (1 - b1^t)) /
(sqrt(v / (1 - b2^t)) + eps).  Parameters are one flat vector laid out as
W1[64][32], b1[64], W2[64][64], b2[64], W3[12][64], b3[12]."""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 32, 64, 12
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)   # 7052


def unpack(p: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[k:k + n].reshape(shape)
        k += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def forward(p: np.ndarray, X: np.ndarray):
    w = unpack(np.asarray(p, np.float64))
    X = np.asarray(X, np.float64)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w["W3"].T + w["b3"]
    return z, (X, a1, h1, a2, h2)


def masked_softmax(z: np.ndarray, mask: np.ndarray) -> np.ndarray:
    zm = np.where(mask, z, -np.inf)
    zm = zm - zm.max(axis=1, keepdims=True)
    e = np.where(mask, np.exp(zm), 0.0)
    return e / e.sum(axis=1, keepdims=True)


def loss_grad(p: np.ndarray, X: np.ndarray, y: np.ndarray, mask: np.ndarray):
    """Mean masked cross-entropy and its gradient (flat, like p)."""
    z, (X, a1, h1, a2, h2) = forward(p, X)
    B = len(y)
    P = masked_softmax(z, mask)
    loss = float(-np.log(P[np.arange(B), y]).mean())
    dz = P.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    w = unpack(np.asarray(p, np.float64))
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = (dz @ w["W3"]) * (a2 > 0)
    g["W2"], g["b2"] = dh2.T @ h1, dh2.sum(0)
    dh1 = (dh2 @ w["W2"]) * (a1 > 0)
    g["W1"], g["b1"] = dh1.T @ X, dh1.sum(0)
    return loss, pack(g)


def adam(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def he_init(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (reference initialisation for tests)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            d[name] = rng.normal(0.0, np.sqrt(2.0 / shape[1]), shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)


def train(X, y, mask, epochs=200, batch=256, lr=1e-3, seed=0, p=None):
    p = he_init(seed) if p is None else p.copy()
    m, v = np.zeros_like(p), np.zeros_like(p)
    rng = np.random.default_rng(seed + 1)
    t = 0
    for _ in range(epochs):
        order = rng.permutation(len(y))
        for s in range(0, len(y), batch):
            idx = order[s:s + batch]
            _, g = loss_grad(p, X[idx], y[idx], mask[idx])
            t += 1
            p, m, v = adam(p, g, m, v, t, lr)
    return p


def predict(p, X, mask) -> np.ndarray:
    z, _ = forward(p, X)
    return np.argmax(np.where(mask, z, -np.inf), axis=1)
