"""TEST INFRASTRUCTURE -- FP64 reference of the learned smoothness detector.

A plain numpy implementation (no batching tricks beyond matrix products) of
the 30 -> 32 -> 32 -> 1 multilayer perceptron the CUDA library trains and
evaluates: ReLU hidden layers, a sigmoid output and the binary cross-entropy
loss, with its gradient derived by hand (back-propagation). Used to check the
GPU training kernels' gradients; pinned itself to central finite differences
(tests/test_oracle_learned.py). Only tests/ and bench.py's checks import it.

Parameter vector layout (shared definition of the data format, not of code):
W1[30][32], b1[32], W2[32][32], b2[32], w3[32], b3 -- 2081 values, with
h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), p = sigmoid(h2 . w3 + b3).
"""
from __future__ import annotations

import numpy as np

NIN, NH = 30, 32
NPARAM = NIN * NH + NH + NH * NH + NH + NH + 1


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (NPARAM,)
    o = 0
    W1 = theta[o:o + NIN * NH].reshape(NIN, NH); o += NIN * NH
    b1 = theta[o:o + NH]; o += NH
    W2 = theta[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = theta[o:o + NH]; o += NH
    w3 = theta[o:o + NH]; o += NH
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def forward(theta, X):
    """Probabilities p[n] and the hidden activations."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    p = 1.0 / (1.0 + np.exp(-z))
    return p, (X, a1, h1, a2, h2, z)


def loss(theta, X, y):
    """Sum over samples of the binary cross-entropy -[y log p + (1-y) log(1-p)],
    written through the logit z for stability: log(1 + e^z) - y z."""
    p, (_, _, _, _, _, z) = forward(theta, X)
    y = np.asarray(y, dtype=np.float64)
    return float(np.sum(np.logaddexp(0.0, z) - y * z))


def grad(theta, X, y):
    """Gradient of loss() with respect to the parameter vector (back-propagation:
    dL/dz = p - y, then through w3, the ReLU masks, W2 and W1)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    p, (X, a1, h1, a2, h2, z) = forward(theta, X)
    y = np.asarray(y, dtype=np.float64)
    dz = p - y                                   # (n,)
    g_w3 = h2.T @ dz
    g_b3 = np.sum(dz)
    dh2 = np.outer(dz, w3) * (a2 > 0.0)          # (n, 32)
    g_W2 = h1.T @ dh2
    g_b2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (a1 > 0.0)
    g_W1 = X.T @ dh1
    g_b1 = dh1.sum(axis=0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), via FP32 as the inference
    path does; returned as float64. Finite inputs only."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, X):
    """Logits of the deployed inference arithmetic: inputs, W1 and W2 rounded to
    bfloat16, products accumulated exactly (FP64 here, FP32 on the device),
    FP32 biases; the first hidden layer is rounded to bfloat16 after its ReLU
    (it is the second product's operand); the output layer reads the second
    hidden layer unrounded with FP32 weights."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    x = bf16_round(X)
    a1 = x @ bf16_round(W1) + b1
    h1 = bf16_round(np.maximum(a1, 0.0))
    a2 = h1 @ bf16_round(W2) + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ w3 + b3


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) at step t >= 1 with gradient g:
    m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
