"""FP64 oracle of the learned vertex-pruning predictor.  Test infrastructure
only (callers: the tests and the CPU baseline leg of the benchmark).

The predictor is not part of the paper: it is a 6 -> 32 -> 32 -> 1
multilayer perceptron (ReLU hidden layers, sigmoid output) that estimates
whether a vertex visit of local moving (Algorithm 4) will move the vertex, so
that visits predicted not to move can be skipped.  This module writes out its
definition plainly in float64 with numpy:

  * parameters are one flat array: W1[32][6], b1[32], W2[32][32], b2[32],
    W3[32], b3 (row-major, output unit first);
  * the product path rounds every parameter to bfloat16 (round to nearest,
    ties to even) before use; ``bf16_round`` is that rounding, written from
    the bfloat16 format (the upper 16 bits of an IEEE float32);
  * h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 . h2 + b3,
    p = 1 / (1 + exp(-z));
  * the training loss is the mean binary cross-entropy
    L = mean(softplus(z) - y z), whose gradient is obtained by the chain rule
    (backpropagation) at the rounded parameters;
  * features of a visit (``features``) are log1p(degree)/16,
    log1p(K_i)/log1p(max K), the fraction of K_i kept inside the vertex's
    community at its last visit, the last visit's best gain scaled by m/K_i
    and clamped to [-1, 1], whether that visit moved the vertex, and the
    iteration's position in the pass (iteration / MAX_ITERATIONS).
"""
import numpy as np

N_IN, N_H = 6, 32
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_H * N_IN
OFF_W2 = OFF_B1 + N_H
OFF_B2 = OFF_W2 + N_H * N_H
OFF_W3 = OFF_B2 + N_H
OFF_B3 = OFF_W3 + N_H
N_PARAMS = OFF_B3 + 1


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even); returns
    float32.  A bfloat16 keeps the sign, the 8 exponent bits and the top 7
    mantissa bits of a float32, i.e. its upper 16 bits: add half a unit of
    the dropped 16 bits (minus one when the kept part is even, so that exact
    halves go to the even neighbour) and truncate.  NaN stays NaN."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + keep_lsb) >> np.uint64(16)) << np.uint64(16)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out).astype(np.float32)


def unpack(params, rounded=True):
    """(W1, b1, W2, b2, W3, b3) in float64 from the flat parameter array:
    the float32 parameters rounded to bfloat16, or (rounded=False) the values
    as given, in float64."""
    p = np.asarray(params)
    if p.shape != (N_PARAMS,):
        raise ValueError("expected %d parameters" % N_PARAMS)
    p = bf16_round(p.astype(np.float32)).astype(np.float64) if rounded else p.astype(np.float64)
    return (p[OFF_W1:OFF_B1].reshape(N_H, N_IN), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(N_H, N_H),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3], p[OFF_B3])


def _layers(params, X, rounded):
    W1, b1, W2, b2, W3, b3 = unpack(params, rounded)
    X = np.asarray(X, dtype=np.float64).reshape(-1, N_IN)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3 + b3
    return X, a1, h1, a2, h2, z


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, X, rounded=True):
    """P(move) of each feature row."""
    return sigmoid(_layers(params, X, rounded)[5])


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def loss(params, X, y, rounded=True):
    """Mean binary cross-entropy of the rows' predictions against y (0/1)."""
    z = _layers(params, X, rounded)[5]
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(softplus(z) - y * z))


def loss_and_grad(params, X, y, rounded=True):
    """(loss, dloss/dparams) by backpropagation through the three layers."""
    W1, b1, W2, b2, W3, b3 = unpack(params, rounded)
    X, a1, h1, a2, h2, z = _layers(params, X, rounded)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    L = float(np.mean(softplus(z) - y * z))
    dz = (sigmoid(z) - y) / n               # dL/dz per row
    g = np.zeros(N_PARAMS)
    g[OFF_B3] = dz.sum()
    g[OFF_W3:OFF_B3] = h2.T @ dz
    da2 = np.outer(dz, W3) * (a2 > 0)       # through relu
    g[OFF_B2:OFF_W3] = da2.sum(axis=0)
    g[OFF_W2:OFF_B2] = (da2.T @ h1).ravel()
    da1 = (da2 @ W2) * (a1 > 0)
    g[OFF_B1:OFF_W2] = da1.sum(axis=0)
    g[OFF_W1:OFF_B1] = (da1.T @ X).ravel()
    return L, g


def features(degree, K, kept, gain, moved, max_K, iteration, max_iterations):
    """Predictor inputs of visits (arrays broadcast together), float64."""
    degree = np.asarray(degree, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    max_logk = np.log1p(max_K)
    if not max_logk > 0:
        max_logk = 1.0
    cols = [np.log1p(degree) / 16.0, np.log1p(K) / max_logk, np.asarray(kept, dtype=np.float64),
            np.asarray(gain, dtype=np.float64), np.asarray(moved, dtype=np.float64),
            np.full(np.broadcast(degree, K).shape, iteration / max_iterations if max_iterations else 0.0)]
    return np.stack(np.broadcast_arrays(*cols), axis=-1)


def adam_step(params, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, 2015, Algorithm 1) in float64: returns the
    new (params, m, v).  t is the 1-based step number."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return np.asarray(params, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
