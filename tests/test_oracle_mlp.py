"""Pins for the FP64 oracle of the learned pruning predictor (oracle/mlp.py),
each against something other than the oracle itself: hand-computed values,
the bfloat16 conversion of a library (torch on the CPU), central finite
differences of the loss, closed forms for degenerate networks, and the
descent property of a gradient step.  CPU only."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp


def rand_params(rng, scale=0.5):
    return (rng.standard_normal(mlp.N_PARAMS) * scale).astype(np.float32)


def rand_rows(rng, n):
    X = np.stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(-1, 1, n),
                  rng.integers(0, 2, n), rng.uniform(0, 1, n)], axis=1)
    y = rng.integers(0, 2, n)
    return X, y


# ------------------------------------------------------------- bfloat16
def test_bf16_round_hand_values():
    one = np.float32(1.0)
    vals = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7 + 2.0 ** -9, -2.5, 0.0, -0.0,
                     np.inf, -np.inf, 3.4e38], dtype=np.float32)
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -2.5, 0.0, -0.0, np.inf, -np.inf, np.inf],
                    dtype=np.float32)
    got = mlp.bf16_round(vals)
    assert np.array_equal(got, want)
    assert np.signbit(got[6])
    assert np.isnan(mlp.bf16_round(np.array([np.nan], np.float32)))[0]
    assert mlp.bf16_round(one) == one


def test_bf16_round_matches_library_conversion():
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[~np.isnan(x)]
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    got = mlp.bf16_round(x)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


# ------------------------------------------------------------- forward
def test_forward_hand_network():
    """A single path x0 -> h1[0] -> h2[0] -> z with unit weights: z = x0 for
    x0 > 0, so p = sigmoid(x0); at x0 = ln 3, p = 3/4."""
    p = np.zeros(mlp.N_PARAMS, np.float32)
    p[mlp.OFF_W1 + 0] = 1.0
    p[mlp.OFF_W2 + 0] = 1.0
    p[mlp.OFF_W3 + 0] = 1.0
    X = np.zeros((3, 6))
    X[0, 0] = math.log(3.0)
    X[1, 0] = -2.0   # relu cuts it: z = 0, p = 1/2
    X[2, 1] = 5.0    # feature 1 is not wired
    got = mlp.forward(p, X)
    assert got[0] == pytest.approx(0.75, rel=1e-6)  # ln 3 is not exact in float64
    assert got[1] == 0.5 and got[2] == 0.5
    # y = (1, 0, 1): loss = mean(-ln 3/4, ln 2, ln 2)
    assert mlp.loss(p, X, [1, 0, 1]) == pytest.approx((-math.log(0.75) + 2 * math.log(2)) / 3, rel=1e-6)


def test_forward_uses_rounded_weights():
    p = np.zeros(mlp.N_PARAMS, np.float32)
    p[mlp.OFF_B3] = np.float32(1 + 2.0 ** -8)  # rounds to 1.0 in bfloat16
    X = np.zeros((1, 6))
    assert mlp.forward(p, X)[0] == pytest.approx(1 / (1 + math.exp(-1.0)), rel=1e-15)
    assert mlp.forward(p, X, rounded=False)[0] == pytest.approx(1 / (1 + math.exp(-(1 + 2.0 ** -8))), rel=1e-15)


def test_zero_output_layer_closed_form():
    """W3 = 0: z = b3 for every row, so p = sigmoid(b3), the loss is
    softplus(b3) - mean(y) b3, dL/db3 = sigmoid(b3) - mean(y) and no gradient
    reaches the hidden layers."""
    rng = np.random.default_rng(1)
    p = rand_params(rng)
    p[mlp.OFF_W3:mlp.OFF_B3] = 0.0
    p[mlp.OFF_B3] = -0.75
    X, y = rand_rows(rng, 500)
    b3 = -0.75
    L, g = mlp.loss_and_grad(p, X, y)
    assert np.allclose(mlp.forward(p, X), 1 / (1 + math.exp(0.75)), rtol=1e-15)
    assert L == pytest.approx(math.log1p(math.exp(b3)) - y.mean() * b3, rel=1e-12)
    assert g[mlp.OFF_B3] == pytest.approx(1 / (1 + math.exp(0.75)) - y.mean(), rel=1e-12)
    assert np.all(g[:mlp.OFF_W3] == 0.0)


# ------------------------------------------------------------- gradient
@pytest.mark.parametrize("seed", [2, 3])
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = rand_params(rng).astype(np.float64)
    X, y = rand_rows(rng, 64)
    _, g = mlp.loss_and_grad(p, X, y, rounded=False)

    def L(q):
        return mlp.loss(q, X, y, rounded=False)

    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 80, replace=False),
                          [mlp.OFF_W1, mlp.OFF_B1, mlp.OFF_W2, mlp.OFF_B2, mlp.OFF_W3, mlp.OFF_B3]])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (L(p + e) - L(p - e)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_gradient_step_descends():
    rng = np.random.default_rng(4)
    p = rand_params(rng)
    X, y = rand_rows(rng, 400)
    L0, g = mlp.loss_and_grad(p, X, y, rounded=False)
    p1 = (p - 1e-3 * g / np.linalg.norm(g)).astype(np.float32)
    assert mlp.loss(p1, X, y, rounded=False) < L0


# ------------------------------------------------------------- features
def test_features_closed_values():
    x = mlp.features(degree=[0, math.e ** 16 - 1], K=[0.0, 7.0], kept=[0.25, 1.0], gain=[-1.0, 0.5],
                     moved=[1, 0], max_K=7.0, iteration=5, max_iterations=20)
    assert x.shape == (2, 6)
    assert np.allclose(x[:, 0], [0.0, 1.0])
    assert np.allclose(x[:, 1], [0.0, 1.0])
    assert np.array_equal(x[:, 2:5], [[0.25, -1.0, 1.0], [1.0, 0.5, 0.0]])
    assert np.all(x[:, 5] == 0.25)


# ------------------------------------------------------------- Adam
def test_adam_first_step_is_signed_learning_rate():
    """At t = 1 the bias corrections undo the zero initial moments: the step
    is lr * g / (|g| + eps), i.e. lr * sign(g) up to eps."""
    rng = np.random.default_rng(5)
    g = rng.standard_normal(mlp.N_PARAMS)
    g[0] = 0.0
    p0 = rng.standard_normal(mlp.N_PARAMS)
    p1, m, v = mlp.adam_step(p0, g, np.zeros_like(g), np.zeros_like(g), lr=0.01, t=1)
    assert np.allclose(p0 - p1, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)
    assert np.allclose(p0 - p1, 0.01 * np.sign(g), rtol=1e-3, atol=0)  # smallest |g| here ~1.5e-5
    assert p1[0] == p0[0]
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_keeps_unit_steps():
    """With a constant gradient the bias-corrected moments equal g and g^2 at
    every step, so every step moves by lr * sign(g)."""
    g = np.array([2.0, -0.5, 1e-3])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 6):
        q, m, v = mlp.adam_step(p, g, m, v, lr=0.1, t=t)
        assert np.allclose(p - q, 0.1 * np.sign(g), rtol=1e-5)
        p = q
