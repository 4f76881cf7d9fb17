"""FP64 oracle of the learned warm start's network (test infrastructure only).

A multilayer perceptron maps one row per (agent, direction, station) -
x = [J_prev (8 reals), (B_f Z_prev) (8 reals), normalised frequency] - to a correction of the
previous interval's Jones matrix: J_init = J_prev + y. The paper initialises each J-update
from the previous time slot's solution (Section 3, initialisation); the network refines that
start and is kept only where it lowers L_i. Written plainly: dense layers, ReLU, mean squared
error, and AdamW (decoupled weight decay), each step in order.

Weights are given as float64 arrays; the GPU computes with bfloat16 copies of its float32
master weights, so tests pass the bfloat16-rounded values here.
"""
from __future__ import annotations

import numpy as np


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, X):
    """params: list of (W [out,in], b [out]); hidden layers use ReLU, the last is linear.
    Returns the output [n, 8] and the list of layer inputs (for backward)."""
    acts = [X]
    h = X
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        h = relu(z) if i < len(params) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grads(params, X, target):
    """Mean over rows of ||J_prev + y - target||^2 and its gradient with respect to every
    weight and bias (reverse-mode chain rule through the dense layers and ReLU)."""
    n = X.shape[0]
    y, acts = forward(params, X)
    pred = X[:, :8] + y
    diff = pred - target
    loss = float(np.sum(diff * diff) / n)
    g = 2.0 * diff / n  # d loss / d y
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, b = params[i]
        h_in = acts[i]
        grads[i] = (g.T @ h_in, g.sum(axis=0))
        if i > 0:
            g = (g @ W) * (acts[i] > 0.0)  # through the ReLU of the layer below
    return loss, grads


def adamw_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step (Loshchilov and Hutter): moments, bias correction, decoupled decay."""
    out = []
    for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, gp) in enumerate(((W, gW), (b, gb))):
            m[i][j] = beta1 * m[i][j] + (1 - beta1) * gp
            v[i][j] = beta2 * v[i][j] + (1 - beta2) * gp * gp
            mh = m[i][j] / (1 - beta1 ** t)
            vh = v[i][j] / (1 - beta2 ** t)
            new.append(p - lr * (mh / (np.sqrt(vh) + eps) + wd * p))
        out.append(tuple(new))
    return out


def features(J_prev, BZ_prev, xf):
    """Rows [A*K*N, 17]: J_prev and B_f Z_prev as (re, im) of the 2x2 row-major entries, and
    the normalised frequency of the row's agent. J_prev, BZ_prev: [A,K,N,2,2]; xf: [A]."""
    A, K, N = J_prev.shape[:3]
    jr = np.stack([J_prev.real, J_prev.imag], -1).reshape(A, K, N, 8)
    br = np.stack([BZ_prev.real, BZ_prev.imag], -1).reshape(A, K, N, 8)
    f = np.broadcast_to(np.asarray(xf, dtype=float)[:, None, None, None], (A, K, N, 1))
    return np.concatenate([jr, br, f], -1).reshape(-1, 17)


def rows_to_jones(Y, A, K, N):
    """Inverse of the J part of features(): [A*K*N, 8] -> complex [A,K,N,2,2]."""
    r = Y.reshape(A, K, N, 2, 2, 2)
    return r[..., 0] + 1j * r[..., 1]
