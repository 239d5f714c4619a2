"""Pins of the FP64 MLP reference: GELU against its definition, backward against finite
differences of the loss (every parameter tensor, masked and unmasked outputs)."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_matches_normal_cdf_definition():
    from scipy.stats import norm
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(mlp.gelu(z), z * norm.cdf(z), atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("masked", [False, True])
def test_backward_matches_finite_differences(masked):
    rng = np.random.default_rng(0)
    dims = [7, 9, 9, 5]
    Ws, bs = mlp.init(dims, rng)
    for b in bs:
        b += 0.1 * rng.standard_normal(b.shape)
    x = rng.standard_normal((6, dims[0]))
    t = rng.standard_normal((6, dims[-1]))
    mask = (rng.uniform(size=dims[-1]) > 0.3).astype(float) if masked else None
    gW, gb = mlp.backward(Ws, bs, x, t, mask)
    h = 1e-6
    for k in range(len(Ws)):
        for idx in [(0, 0), (dims[k + 1] - 1, dims[k] - 1), (1, 2)]:
            W2 = [w.copy() for w in Ws]
            W2[k][idx] += h
            lp = mlp.loss(W2, bs, x, t, mask)
            W2[k][idx] -= 2 * h
            lm = mlp.loss(W2, bs, x, t, mask)
            assert abs((lp - lm) / (2 * h) - gW[k][idx]) < 1e-7
        for j in [0, dims[k + 1] - 1]:
            b2 = [b.copy() for b in bs]
            b2[k][j] += h
            lp = mlp.loss(Ws, b2, x, t, mask)
            b2[k][j] -= 2 * h
            lm = mlp.loss(Ws, b2, x, t, mask)
            assert abs((lp - lm) / (2 * h) - gb[k][j]) < 1e-7
