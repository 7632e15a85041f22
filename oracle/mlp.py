"""Float64 reference of the cut-scoring MLP (64 -> 256 -> 256 -> 1).

The network: h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3,
loss = mean over the batch of (y - t)^2.  Weights W_l are [fan_in][fan_out].
Gradients are the textbook backpropagation of that loss; Adam is the
Kingma-Ba update with bias correction.

The paper has no learned component; this is the reference for the cut
scorer's hand-written kernels.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

SIZES = (64, 256, 256, 1)


def forward(params, x):
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0)
    y = h2 @ W3 + b3
    return y[:, 0], (x, z1, h1, z2, h2)


def loss(params, x, t):
    y, _ = forward(params, x)
    return float(np.mean((y - t) ** 2))


def backward(params, x, t):
    """Gradients of the mean squared error w.r.t. (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    y, (x, z1, h1, z2, h2) = forward(params, x)
    B = x.shape[0]
    dy = (2.0 / B) * (y - t)[:, None]              # [B, 1]
    dW3 = h2.T @ dy
    db3 = dy.sum(axis=0)
    dh2 = dy @ W3.T
    dz2 = dh2 * (z2 > 0)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (z1 > 0)
    dW1 = x.T @ dz1
    db1 = dz1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = beta1 * mm + (1 - beta1) * g
        vv = beta2 * vv + (1 - beta2) * g * g
        mh = mm / (1 - beta1 ** step)
        vh = vv / (1 - beta2 ** step)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
