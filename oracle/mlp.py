"""fp64 CPU oracle of the learned-scheduler MLP — test infrastructure only.

The network is not from the paper (the paper only asks for an adaptive runtime
choice of solver, Sec. 5 and the conclusion); it is the scheduler network of this
library: features -> 64 -> 64 -> logits of three softmax heads
(sweep mode, bucket-width class, block configuration), ReLU activations, loss
= mean over the batch of the sum over heads of the softmax cross-entropy.

Parameter layout (row-major, fp32 on the device, fp64 here):
    W1[F, H1], b1[H1], W2[H1, H2], b2[H2], W3[H2, O], b3[O]
flattened in that order into one vector.  Heads are contiguous slices of the O
logits given by ``heads`` (sizes).  Pinned in tests by central finite
differences of ``loss`` against ``backward``, by a hand-worked forward pass
with nonzero weights and clipped units, and by three hand-worked Adam steps
(bias corrections at t = 1, 2, 3).
"""
from __future__ import annotations

import numpy as np


def shapes(F: int, H1: int, H2: int, O: int):
    return [(F, H1), (H1,), (H1, H2), (H2,), (H2, O), (O,)]


def unflatten(theta: np.ndarray, F: int, H1: int, H2: int, O: int):
    out, k = [], 0
    for s in shapes(F, H1, H2, O):
        sz = int(np.prod(s))
        out.append(theta[k:k + sz].reshape(s))
        k += sz
    return out


def forward(theta, X, F, H1, H2, O):
    W1, b1, W2, b2, W3, b3 = unflatten(np.asarray(theta, np.float64), F, H1, H2, O)
    X = np.asarray(X, np.float64)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3 + b3
    return z, (X, a1, h1, a2, h2)


def _head_slices(heads):
    s, out = 0, []
    for h in heads:
        out.append(slice(s, s + h))
        s += h
    return out


def loss(theta, X, Y, heads, F, H1, H2, O) -> float:
    """Y int[B, len(heads)] class labels per head."""
    z, _ = forward(theta, X, F, H1, H2, O)
    B = z.shape[0]
    tot = 0.0
    for j, sl in enumerate(_head_slices(heads)):
        zh = z[:, sl]
        mx = zh.max(axis=1, keepdims=True)
        lse = mx[:, 0] + np.log(np.exp(zh - mx).sum(axis=1))
        tot += float((lse - zh[np.arange(B), Y[:, j]]).sum())
    return tot / B


def backward(theta, X, Y, heads, F, H1, H2, O):
    """Returns (loss, gradient vector with the layout of theta)."""
    theta = np.asarray(theta, np.float64)
    W1, b1, W2, b2, W3, b3 = unflatten(theta, F, H1, H2, O)
    z, (X, a1, h1, a2, h2) = forward(theta, X, F, H1, H2, O)
    B = z.shape[0]
    dz = np.zeros_like(z)
    tot = 0.0
    for j, sl in enumerate(_head_slices(heads)):
        zh = z[:, sl]
        mx = zh.max(axis=1, keepdims=True)
        e = np.exp(zh - mx)
        p = e / e.sum(axis=1, keepdims=True)
        tot += float((np.log(e.sum(axis=1)) + mx[:, 0] - zh[np.arange(B), Y[:, j]]).sum())
        p[np.arange(B), Y[:, j]] -= 1.0
        dz[:, sl] = p / B
    gW3 = h2.T @ dz
    gb3 = dz.sum(axis=0)
    dh2 = dz @ W3.T
    da2 = dh2 * (a2 > 0)
    gW2 = h1.T @ da2
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2.T
    da1 = dh1 * (a1 > 0)
    gW1 = X.T @ da1
    gb1 = da1.sum(axis=0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return tot / B, g


def adam_step(theta, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba 2015), bias-corrected with step count t >= 1."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def predict(theta, X, heads, F, H1, H2, O):
    z, _ = forward(theta, X, F, H1, H2, O)
    return np.stack([z[:, sl].argmax(axis=1) for sl in _head_slices(heads)], axis=1)
