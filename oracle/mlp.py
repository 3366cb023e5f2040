"""FP64 oracle for the per-area warm-start MLP (not part of the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network: Linear -> GELU -> Linear -> GELU -> Linear -> GELU -> Linear, i.e.
three hidden layers, with GELU in its exact erf form
gelu(u) = u * Phi(u) = 0.5 * u * (1 + erf(u / sqrt(2))).
Layer l maps a row vector a (batch-major, [B, d_in]) to a @ W_l^T + b_l with
W_l stored [d_out, d_in].
Loss: mean squared error over batch and outputs,
loss = sum((y_hat - y)^2) / (B * d_out).
Update: AdamW with decoupled weight decay: p <- p * (1 - lr * wd), then
p <- p - lr * m_hat / (sqrt(v_hat) + eps) with bias-corrected moments.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

_SQRT2 = math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(u):
    return 0.5 * u * (1.0 + erf(u / _SQRT2))


def gelu_grad(u):
    """d gelu / du = Phi(u) + u * phi(u)."""
    return 0.5 * (1.0 + erf(u / _SQRT2)) + u * _INV_SQRT_2PI * np.exp(-0.5 * u * u)


def forward(params, X):
    """Returns (pre-activations, activations, output).  params = [(W, b), ...]."""
    a = np.asarray(X, dtype=float)
    pre, acts = [], [a]
    for li, (W, b) in enumerate(params):
        u = a @ W.T + b
        pre.append(u)
        a = gelu(u) if li + 1 < len(params) else u
        acts.append(a)
    return pre, acts, a


def loss_and_grads(params, X, Y):
    """MSE loss and its gradients w.r.t. every (W, b), by backpropagation."""
    pre, acts, out = forward(params, X)
    B, d_out = out.shape
    diff = out - Y
    loss = float(np.sum(diff * diff) / (B * d_out))
    delta = 2.0 * diff / (B * d_out)              # dloss/d(output)
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        grads[li] = (delta.T @ acts[li], delta.sum(axis=0))
        if li > 0:
            delta = (delta @ W) * gelu_grad(pre[li - 1])
    return loss, grads


def adamw_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update of array p in place; returns (m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    p *= (1.0 - lr * wd)
    p -= lr * mhat / (np.sqrt(vhat) + eps)
    return m, v
