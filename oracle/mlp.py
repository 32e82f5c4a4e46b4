"""CPU oracle of the controller network (FP64).  TEST INFRASTRUCTURE ONLY.

12 -> 64 (ReLU) -> 64 (ReLU) -> 9 outputs; loss = CE(m head, outputs 0..2) + (y3 - tl)^2 +
CE(d head, outputs 4..7) + (y8 - rt)^2, each term averaged over the batch; a class label of -1
(or any value outside the head's classes) drops that sample's cross-entropy term.  Parameters in the library's flat order:
W1[64][12], b1[64], W2[64][64], b2[64], W3[9][64], b3[9].
"""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (64, 12)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (9, 64)),
          ("b3", (9,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, off = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[off:off + k], dtype=np.float64).reshape(shape)
        off += k
    return out


def forward(p, X):
    w = unpack(p)
    X = np.asarray(X, np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["W3"].T + w["b3"]
    return y, (X, z1, h1, z2, h2)


def _ce(logits, labels):
    """Mean-over-batch cross-entropy terms and d(loss)/d(logits) (already divided by B)."""
    B = logits.shape[0]
    mx = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - mx)
    p = e / e.sum(axis=1, keepdims=True)
    loss = np.zeros(B)
    d = np.zeros_like(logits)
    for b in range(B):
        if labels[b] < 0 or labels[b] >= logits.shape[1]:
            continue
        loss[b] = -np.log(p[b, labels[b]])
        d[b] = p[b]
        d[b, labels[b]] -= 1.0
    return loss.mean(), d / B


def loss_and_grad(p, X, mc, tl, dc, rt):
    """The four batch-mean loss terms and the gradient of their sum."""
    w = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    B = X.shape[0]
    l0, d0 = _ce(y[:, 0:3], mc)
    l2, d2 = _ce(y[:, 4:8], dc)
    e3 = y[:, 3] - tl
    e8 = y[:, 8] - rt
    dy = np.zeros_like(y)
    dy[:, 0:3] = d0
    dy[:, 4:8] = d2
    dy[:, 3] = 2 * e3 / B
    dy[:, 8] = 2 * e8 / B
    losses = np.array([l0, np.mean(e3 ** 2), l2, np.mean(e8 ** 2)])
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = (dy @ w["W3"]) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ w["W2"]) * (z1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return losses, g
