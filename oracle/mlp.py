"""A 3-layer perceptron, its gradient and one Adam step, in plain FP64 numpy (oracle, test-only).

Network (width H, inputs F, outputs O), for a batch X (N x F):
  Z1 = X W1^T + b1,  A1 = tanh(Z1)        W1: H x F
  Z2 = A1 W2^T + b2, A2 = tanh(Z2)        W2: H x H
  Y  = A2 W3^T + b3                       W3: O x H
Loss: L = sum over samples and outputs of (Y - T)^2 / (N O)  (mean squared error).
Gradients by the chain rule (d tanh(z)/dz = 1 - tanh(z)^2), written out layer by layer.
Adam (Kingma and Ba, ICLR 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Packed parameter order (one flat vector): W1 (row-major), b1, W2, b2, W3, b3.
"""
from __future__ import annotations

import numpy as np


def shapes(F: int, H: int, O: int):
    return [(H, F), (H,), (H, H), (H,), (O, H), (O,)]


def n_params(F: int, H: int, O: int) -> int:
    return sum(int(np.prod(s)) for s in shapes(F, H, O))


def unpack(theta: np.ndarray, F: int, H: int, O: int):
    out, off = [], 0
    for s in shapes(F, H, O):
        size = int(np.prod(s))
        out.append(theta[off:off + size].reshape(s))
        off += size
    return out


def forward(theta, X, F, H, O):
    """Y and the activations (A1, A2) of the batch X."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64), F, H, O)
    X = np.asarray(X, dtype=np.float64)
    A1 = np.tanh(X @ W1.T + b1)
    A2 = np.tanh(A1 @ W2.T + b2)
    Y = A2 @ W3.T + b3
    return Y, A1, A2


def loss(theta, X, T, F, H, O) -> float:
    Y, _, _ = forward(theta, X, F, H, O)
    return float(np.mean((Y - np.asarray(T, dtype=np.float64)) ** 2))


def gradient(theta, X, T, F, H, O):
    """(L, dL/dtheta) in the packed order."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64), F, H, O)
    X = np.asarray(X, dtype=np.float64)
    Y, A1, A2 = forward(theta, X, F, H, O)
    N = X.shape[0]
    D = Y - np.asarray(T, dtype=np.float64)
    L = float(np.mean(D ** 2))
    dY = 2.0 * D / (N * O)                 # dL/dY
    dW3 = dY.T @ A2
    db3 = dY.sum(axis=0)
    dA2 = dY @ W3
    dZ2 = dA2 * (1.0 - A2 ** 2)
    dW2 = dZ2.T @ A1
    db2 = dZ2.sum(axis=0)
    dA1 = dZ2 @ W2
    dZ1 = dA1 * (1.0 - A1 ** 2)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return L, g


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
