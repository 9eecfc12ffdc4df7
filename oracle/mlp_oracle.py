"""FP64 CPU oracle of the learned (tau, m) controller network.

TEST INFRASTRUCTURE ONLY (tests, smoke(), bench.py's CPU baseline); never the
product path.

The network is the one the task specifies for the learned controller: 8 inputs,
two hidden layers of 64 GELU units, 2 outputs, trained by mean squared error
with Adam.  This module is its plain definition, written out:

  z1 = W1 x + b1,  h1 = gelu(z1),  z2 = W2 h1 + b2,  h2 = gelu(z2),  y = W3 h2 + b3
  gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2          (exact, erf-based)
  loss = mean over rows and outputs of (y - target)^2
  Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
      w -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)

Parameter vector layout (shared with the CUDA kernels as an interface):
  W1 [64 x 8] row-major at 0, b1 [64] at 512, W2 [64 x 64] at 576, b2 [64] at 4672,
  W3 [2 x 64] at 4736, b3 [2] at 4864; 4866 values.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H, N_OUT = 8, 64, 2
OFF_W1, OFF_B1 = 0, 512
OFF_W2, OFF_B2 = 576, 4672
OFF_W3, OFF_B3 = 4736, 4864
N_PARAMS = 4866

_erf = np.vectorize(math.erf)


def unpack(w: np.ndarray):
    w = np.asarray(w, dtype=np.float64)
    W1 = w[OFF_W1:OFF_B1].reshape(N_H, N_IN)
    b1 = w[OFF_B1:OFF_W2]
    W2 = w[OFF_W2:OFF_B2].reshape(N_H, N_H)
    b2 = w[OFF_B2:OFF_W3]
    W3 = w[OFF_W3:OFF_B3].reshape(N_OUT, N_H)
    b3 = w[OFF_B3:N_PARAMS]
    return W1, b1, W2, b2, W3, b3


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(w, X):
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(w, X, T):
    """Mean squared error over all rows and outputs, and its gradient (4866 values)."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    y, (X, z1, h1, z2, h2) = forward(w, X)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    r = y - T
    loss = float(np.sum(r * r) / (n * N_OUT))
    dy = 2.0 * r / (n * N_OUT)
    g = np.zeros(N_PARAMS)
    g[OFF_W3:OFF_B3] = (dy.T @ h2).ravel()
    g[OFF_B3:N_PARAMS] = dy.sum(axis=0)
    dz2 = (dy @ W3) * gelu_grad(z2)
    g[OFF_W2:OFF_B2] = (dz2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    g[OFF_W1:OFF_B1] = (dz1.T @ X).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    return loss, g


def adam_step(w, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def init_weights(seed: int) -> np.ndarray:
    """Scaled uniform initialisation (He-style fan-in bound), deterministic from seed."""
    from paper_0907_4631_gb300 import workloads as wl
    w = np.zeros(N_PARAMS)
    w[OFF_W1:OFF_B1] = wl.uniform(seed, 1, 512, -1.0, 1.0) * math.sqrt(6.0 / N_IN)
    w[OFF_W2:OFF_B2] = wl.uniform(seed, 2, 4096, -1.0, 1.0) * math.sqrt(6.0 / N_H)
    w[OFF_W3:OFF_B3] = wl.uniform(seed, 3, 128, -1.0, 1.0) * math.sqrt(6.0 / N_H) * 0.1
    return w
