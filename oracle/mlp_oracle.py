"""FP64 CPU oracle of the learned extrapolation proposer's network.

TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only the test suite may import
this module.  (The proposer has no counterpart in the paper: it chooses the
beta of eq. 19 and is judged against the Section 4.2 rule.)

Network: F -> H -> H -> H -> C, ReLU after every hidden layer, softmax
cross-entropy loss averaged over the batch.  Parameters are one flat vector
holding, for each layer, the weight matrix (out x in, row-major) followed by
the bias.  Forward and backward are written out layer by layer.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

F, H, C = 32, 128, 8
SHAPES = [(H, F), (H, H), (H, H), (C, H)]
NPARAMS = sum(o * i + o for o, i in SHAPES)


def unpack(params: np.ndarray) -> List[Tuple[np.ndarray, np.ndarray]]:
    out, off = [], 0
    p = np.asarray(params, dtype=np.float64)
    for o, i in SHAPES:
        W = p[off:off + o * i].reshape(o, i)
        off += o * i
        b = p[off:off + o]
        off += o
        out.append((W, b))
    assert off == NPARAMS
    return out


def forward(params, X, store=None):
    """Returns logits and the list of layer inputs (post-ReLU activations).

    ``store`` (optional) maps each hidden activation to the values a kernel keeps in
    memory (e.g. rounding to bf16); the next layer and the backward pass use those."""
    layers = unpack(params)
    h = np.asarray(X, dtype=np.float64)
    acts = [h]
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        if l < len(layers) - 1:
            h = np.maximum(z, 0.0)
            if store is not None:
                h = store(h)
            acts.append(h)
        else:
            return z, acts
    raise AssertionError


def bf16(a):
    """Round to the nearest bf16 value (ties to even) through float32, returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grad(params, X, y, store=None):
    """Mean softmax cross-entropy and its gradient (flat, same packing as params)."""
    layers = unpack(params)
    logits, acts = forward(params, X, store)
    B = logits.shape[0]
    z = logits - logits.max(axis=1, keepdims=True)
    p = np.exp(z)
    p /= p.sum(axis=1, keepdims=True)
    y = np.asarray(y, dtype=np.int64)
    loss = float(np.mean(-np.log(p[np.arange(B), y])))
    dz = p.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a = acts[l]
        grads[l] = (dz.T @ a, dz.sum(axis=0))
        if l > 0:
            dz = (dz @ W) * (a > 0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases."""
    g = np.random.default_rng(seed)
    parts = []
    for o, i in SHAPES:
        parts.append(g.standard_normal(o * i) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def adam_step(w, m_, v, g, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba, 2015) with bias correction; returns new (w, m, v)."""
    m_ = b1 * m_ + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m_ / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m_, v
