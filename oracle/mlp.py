"""FP64 reference of the warm-start MLP (test infrastructure only, see ``oracle/__init__``).

Network: x -> [Linear -> GELU] x L -> Linear -> y, GELU(z) = z Phi(z) with the exact normal CDF
Phi(z) = (1 + erf(z / sqrt 2)) / 2.  Loss: mean over the batch and the unmasked outputs of the
squared error.  Weights are stored (out_features, in_features) like the CUDA path.

``forward`` and ``backward`` are written out layer by layer (chain rule by hand); the tests pin
``backward`` against central finite differences of ``loss``.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(weights, biases, x):
    """Returns the output and the per-layer (input, pre-activation) cache."""
    h = x
    cache = []
    n = len(weights)
    for k, (W, b) in enumerate(zip(weights, biases)):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if k < n - 1 else z
    return h, cache


def loss(weights, biases, x, target, mask=None):
    y, _ = forward(weights, biases, x)
    d = y - target
    if mask is not None:
        d = d * mask
        count = x.shape[0] * float(np.sum(mask))
    else:
        count = float(d.size)
    return float(np.sum(d * d) / count)


def backward(weights, biases, x, target, mask=None):
    """Gradients of ``loss`` with respect to every weight matrix and bias vector."""
    y, cache = forward(weights, biases, x)
    d = y - target
    if mask is not None:
        d = d * mask
        count = x.shape[0] * float(np.sum(mask))
    else:
        count = float(d.size)
    g = 2.0 * d / count                      # dL/dy
    gW, gb = [None] * len(weights), [None] * len(weights)
    for k in range(len(weights) - 1, -1, -1):
        h_in, z = cache[k]
        if k < len(weights) - 1:
            g = g * gelu_grad(z)             # through the activation of layer k
        gW[k] = g.T @ h_in
        gb[k] = g.sum(axis=0)
        g = g @ weights[k]                   # dL/dh_in
    return gW, gb


def init(dims, rng):
    """He-style init: W ~ N(0, 2 / fan_in), b = 0."""
    Ws, bs = [], []
    for fin, fout in zip(dims[:-1], dims[1:]):
        Ws.append(rng.standard_normal((fout, fin)) * math.sqrt(2.0 / fin))
        bs.append(np.zeros(fout))
    return Ws, bs
