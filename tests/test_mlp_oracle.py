"""Pins of the planner-network oracle (oracle/mlp.py), CPU only."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_against_definition():
    # values exactly representable in BF16 stay; halfway cases go to even
    exact = np.array([0.0, 1.0, -2.5, 2.0 ** 127, 1.5 * 2.0 ** 100, 2.0 ** -126], dtype=np.float32)
    assert np.array_equal(mlp.bf16(exact), exact.astype(np.float64))
    one = np.float32(1.0)
    ulp = 2.0 ** -7                      # BF16 spacing at 1.0
    assert mlp.bf16(np.float32(1.0 + ulp / 2))[()] == 1.0            # tie -> even (1.0)
    assert mlp.bf16(np.float32(1.0 + 3 * ulp / 2))[()] == 1.0 + 2 * ulp   # tie -> even
    assert mlp.bf16(np.float32(1.0 + ulp / 2 + 2 ** -20))[()] == 1.0 + ulp
    assert one == 1.0


def test_gradient_matches_finite_differences():
    """Central differences of the unrounded float64 loss at a random point."""
    g = np.random.default_rng(0)
    p = mlp.init_params(1).astype(np.float64) + g.normal(0, 0.01, mlp.NPARAM)
    X = g.normal(size=(16, mlp.NIN))
    T = g.normal(size=(16, mlp.NOUT))
    M = (g.random((16, mlp.NOUT)) < 0.8).astype(np.float64)
    loss, grad = mlp.loss_and_grad(p, X, T, M, round_bf16=False)
    idx = g.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, T, M, False)[0] - mlp.loss_and_grad(pm, X, T, M, False)[0]) / (2 * h)
        assert fd == pytest.approx(grad[i], rel=1e-4, abs=1e-8)


def test_forward_shapes_and_layout():
    p = mlp.init_params(3)
    assert p.size == mlp.NPARAM == 24 * 128 + 128 + 128 * 128 + 128 + 128 * 3 + 3
    W = mlp.unpack(p)
    X = np.zeros((5, 24))
    # zero input: the output is the network applied to the biases only
    y = mlp.forward(p, X, round_bf16=False)[3]
    h1 = np.maximum(W["b1"], 0)
    h2 = np.maximum(h1 @ W["W2"] + W["b2"], 0)
    assert np.allclose(y, np.tile(h2 @ W["W3"] + W["b3"], (5, 1)))
