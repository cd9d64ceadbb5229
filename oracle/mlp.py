"""CPU ORACLE (test infrastructure only): the format selector network in float64.

Sec. V-A/V-B: a classifier trained offline on (features, best-format label)
pairs; Sec. V-B "Feature Scaling": every feature is mapped to [0, 1] with the
training set's per-feature minimum and maximum, which are stored with the
model and reused on new matrices.  Sec. V-D lists a multilayer perceptron
among the alternatives; this library's selector is one:

    t   = transform(f)                       (log2(1+f) for size/count features,
                                              -log2(max(f, 2^-60)) for nnz_frac)
    x   = clamp((t - lo) / (hi - lo), 0, 1)  (0 where hi == lo)
    h1  = relu(x  W1 + b1)                   W1: 16 x 64
    h2  = relu(h1 W2 + b2)                   W2: 64 x 64
    z   = h2 W3 + b3                         W3: 64 x 5
    p   = softmax(z);  loss = mean_b -log p[b, label_b]
    prediction = argmax z

Parameters are one flat vector, row-major matrices in the order
W1, b1, W2, b2, W3, b3 (5,573 values).  Adam (Kingma & Ba) updates them.
"""
from __future__ import annotations

import numpy as np

N_FEAT, H1, H2, N_CLASS = 16, 64, 64, 5
SHAPES = (("W1", (N_FEAT, H1)), ("b1", (H1,)), ("W2", (H1, H2)), ("b2", (H2,)), ("W3", (H2, N_CLASS)), ("b3", (N_CLASS,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 5573
LOG_FEATURES = (0, 1, 3, 4, 5, 6, 11, 12)
NNZ_FRAC = 2


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def transform(f: np.ndarray) -> np.ndarray:
    """Feature transform before min-max scaling (float64, any leading shape)."""
    t = np.array(f, dtype=np.float64, copy=True)
    for j in LOG_FEATURES:
        t[..., j] = np.log2(1.0 + t[..., j])
    t[..., NNZ_FRAC] = -np.log2(np.maximum(t[..., NNZ_FRAC], 2.0 ** -60))
    return t


def fit_scaling(t: np.ndarray):
    """Per-feature minimum and maximum over the training rows of transformed features."""
    return t.min(axis=0), t.max(axis=0)


def scale(t: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    span = hi - lo
    safe = np.where(span > 0, span, 1.0)
    x = np.where(span > 0, (t - lo) / safe, 0.0)
    return np.clip(x, 0.0, 1.0)


def forward(theta: np.ndarray, x: np.ndarray):
    p = unpack(theta)
    a1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"] + p["b3"]
    return z, (x, a1, h1, a2, h2)


def softmax(z: np.ndarray) -> np.ndarray:
    e = np.exp(z - z.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def loss(theta: np.ndarray, x: np.ndarray, labels: np.ndarray) -> float:
    z, _ = forward(theta, x)
    pr = softmax(z)
    return float(-np.mean(np.log(pr[np.arange(len(labels)), labels])))


def loss_and_grad(theta: np.ndarray, x: np.ndarray, labels: np.ndarray):
    """Mean cross-entropy and its gradient by backpropagation."""
    z, (x0, a1, h1, a2, h2) = forward(theta, x)
    p = unpack(theta)
    b = x.shape[0]
    pr = softmax(z)
    lval = float(-np.mean(np.log(pr[np.arange(b), labels])))
    dz = pr.copy()
    dz[np.arange(b), labels] -= 1.0
    dz /= b
    g = {"W3": h2.T @ dz, "b3": dz.sum(axis=0)}
    dh2 = dz @ p["W3"].T
    da2 = dh2 * (a2 > 0)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"].T
    da1 = dh1 * (a1 > 0)
    g["W1"] = x0.T @ da1
    g["b1"] = da1.sum(axis=0)
    return lval, pack(g)


def adam_step(theta, grad, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def glorot_init(u: np.ndarray) -> np.ndarray:
    """Map N_PARAMS uniforms in [-1, 1) to Glorot-uniform weights and zero biases."""
    p, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        if len(shape) == 2:
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            p[name] = (u[o:o + k] * lim).reshape(shape)
        else:
            p[name] = np.zeros(shape)
        o += k
    return pack(p)


def predict(theta: np.ndarray, x: np.ndarray) -> np.ndarray:
    z, _ = forward(theta, x)
    return np.argmax(z, axis=-1)
