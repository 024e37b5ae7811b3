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


def _hand_network():
    """A network whose output is worked out by hand: only a few weights are
    non-zero, every value is exactly representable in BF16, and the entries
    sit at asymmetric positions so that a transposed weight matrix, a swapped
    layer, a missing or extra ReLU or a dropped bias changes the output."""
    W = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    W["W1"][0, 5] = 1.0       # input 0 -> hidden-1 unit 5
    W["W1"][1, 5] = 0.5       # input 1 -> hidden-1 unit 5
    W["W1"][1, 9] = -1.0      # input 1 -> hidden-1 unit 9 (negative: cut by the ReLU)
    W["b1"][9] = 0.25
    W["b1"][17] = 2.0         # unit 17: bias only
    W["W2"][5, 3] = 3.0       # hidden-1 unit 5 -> hidden-2 unit 3
    W["W2"][17, 3] = -0.5
    W["W2"][9, 40] = 7.0      # unit 9 is 0 after its ReLU, so unit 40 gets only its bias
    W["b2"][40] = -1.0        # ... which is negative: unit 40 is cut as well
    W["b2"][3] = 0.125
    W["W2"][9, 50] = -2.0     # unit 50 sees unit 9 only after its ReLU (0 here, 7.5 without it)
    W["W3"][3, 0] = 2.0
    W["W3"][3, 2] = -1.0      # a negative output: no ReLU on the last layer
    W["W3"][40, 1] = 100.0    # would show up if unit 40 survived
    W["W3"][50, 0] = 1.0
    W["b3"][:] = [0.5, -0.25, 1.0]
    return np.concatenate([W[name].ravel() for name, _ in mlp.SIZES])


def test_forward_hand_worked_network():
    """x = (2, 4, 0, ...):
    hidden 1: unit 5 = 1*2 + 0.5*4 = 4; unit 9 = relu(-4 + 0.25) = 0; unit 17 = 2.
    hidden 2: unit 3 = 3*4 - 0.5*2 + 0.125 = 11.125; unit 40 = relu(7*0 - 1) = 0;
    unit 50 = relu(-2*0) = 0.
    output: (2*11.125 + 0.5, 0 - 0.25, -11.125 + 1) = (22.75, -0.25, -10.125)."""
    p = _hand_network()
    X = np.zeros((2, mlp.NIN))
    X[0, 0], X[0, 1] = 2.0, 4.0
    y = mlp.forward(p, X)[3]
    assert np.array_equal(y[0], [22.75, -0.25, -10.125])
    # zero input: hidden 1 unit 9 = 0.25, unit 17 = 2; hidden 2 unit 3 = -1 + 0.125 -> 0,
    # unit 40 = relu(7*0.25 - 1) = 0.75, unit 50 = relu(-2*0.25) = 0;
    # output = (0.5, 75 - 0.25, 1.0)
    assert np.array_equal(y[1], [0.5, 74.75, 1.0])


def test_forward_matches_per_neuron_loops():
    """The definition neuron by neuron in plain Python floats (each sum in
    float64, ReLU on the hidden layers only, BF16 rounding of inputs, weights
    and hidden activations) against the vectorised oracle."""
    g = np.random.default_rng(11)
    p = mlp.init_params(12).astype(np.float64) + g.normal(0, 0.05, mlp.NPARAM)
    X = g.normal(size=(3, mlp.NIN))
    r = lambda v: float(mlp.bf16(np.float32(v))[()])
    W = mlp.unpack(mlp.bf16(p))
    want = np.zeros((3, mlp.NOUT))
    for n in range(3):
        x = [r(v) for v in X[n]]
        h1 = []
        for j in range(mlp.NH):
            s = W["b1"][j]
            for i in range(mlp.NIN):
                s += x[i] * W["W1"][i, j]
            h1.append(r(max(s, 0.0)))
        h2 = []
        for j in range(mlp.NH):
            s = W["b2"][j]
            for i in range(mlp.NH):
                s += h1[i] * W["W2"][i, j]
            h2.append(r(max(s, 0.0)))
        for k in range(mlp.NOUT):
            s = W["b3"][k]
            for i in range(mlp.NH):
                s += h2[i] * W["W3"][i, k]
            want[n, k] = s
    got = mlp.forward(p, X)[3]
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
