"""FP64 reference of the ln xi surrogate network: forward, backward, Adam.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU legs); the GPU
library shares nothing with it.

The paper announces a learned selection term that keeps spin effects in VT at
no extra run-time cost (Sec. "Population acceleration", the sentence after the
Monte Carlo VT).  The network here: normalised Lambda (12 inputs) -> four
hidden layers of 256 with SiLU -> 2 outputs (standardised ln xi and ln N_eff).
Parameters are a list of (W [out, in], b [out]).

Loss (per batch of B rows): L = (1/B) sum_b sum_o (y_bo - t_bo)^2.
Backward is the chain rule written out layer by layer; SiLU(z) = z s(z),
SiLU'(z) = s(z) (1 + z (1 - s(z))), s the logistic function.
Adam: Kingma & Ba (2015), bias-corrected moments.
"""
from __future__ import annotations

import numpy as np

LAYERS = (12, 256, 256, 256, 256, 2)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, round_fn=None):
    """Outputs [B, 2] and the per-layer cache (inputs and pre-activations).

    ``round_fn`` (optional) is applied to every hidden activation, to mirror a
    network that stores its activations in a narrower format.
    """
    h = x
    cache = []
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        if li < len(params) - 1:
            h = silu(z)
            if round_fn is not None:
                h = round_fn(h)
        else:
            h = z
    return h, cache


def loss_and_grads(params, x, t, round_fn=None):
    """Mean-squared loss and its gradients [(dW, db), ...] by the chain rule."""
    y, cache = forward(params, x, round_fn)
    B = x.shape[0]
    r = y - t
    loss = float(np.sum(r * r) / B)
    dz = 2.0 * r / B
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        h, z = cache[li]
        W, _ = params[li]
        grads[li] = (dz.T @ h, dz.sum(axis=0))
        if li > 0:
            dh = dz @ W
            dz = dh * dsilu(cache[li - 1][1])
    return loss, grads


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (dW, db), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for p, g, mm, vv in ((W, dW, mW, vW), (b, db, mb, vb)):
            mm = beta1 * mm + (1 - beta1) * g
            vv = beta2 * vv + (1 - beta2) * g * g
            mh = mm / (1 - beta1 ** step)
            vh = vv / (1 - beta2 ** step)
            new.append((p - lr * mh / (np.sqrt(vh) + eps), mm, vv))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v


def zeros_like(params):
    return [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]


def flatten(params):
    """Flat vector in the library's layout: W0, b0, W1, b1, ... (W row-major [out, in])."""
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(vec, layers=LAYERS):
    out, k = [], 0
    for i in range(len(layers) - 1):
        n_in, n_out = layers[i], layers[i + 1]
        W = vec[k:k + n_out * n_in].reshape(n_out, n_in)
        k += n_out * n_in
        b = vec[k:k + n_out]
        k += n_out
        out.append((W.astype(np.float64), b.astype(np.float64)))
    return out


def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
