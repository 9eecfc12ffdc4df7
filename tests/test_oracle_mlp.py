"""Pins of the controller-network oracle: GELU closed forms, the backward pass
against central finite differences, and Adam against a hand-computed step."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_0907_4631_gb300 import workloads as wl


def test_gelu_closed_forms():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    z = np.array([-3.0, -0.5, 0.7, 4.0])
    assert np.allclose(M.gelu(z) - M.gelu(-z), z, rtol=0, atol=1e-15)      # z Phi(z) - (-z) Phi(-z) = z
    assert M.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-14)   # Phi(1)
    h = 1e-6
    for x in [-2.0, -0.3, 0.0, 0.9, 2.5]:
        fd = (M.gelu(np.array([x + h]))[0] - M.gelu(np.array([x - h]))[0]) / (2 * h)
        assert M.gelu_grad(np.array([x]))[0] == pytest.approx(fd, rel=1e-8, abs=1e-10)


def test_layout():
    assert M.N_PARAMS == 8 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2 == 4866


def test_backward_matches_finite_differences():
    w = M.init_weights(5)
    w[M.OFF_B1:M.OFF_W2] = wl.normal(5, 7, 64) * 0.1
    X = wl.normal(6, 1, 7 * 8).reshape(7, 8)
    T = wl.normal(6, 2, 14).reshape(7, 2)
    loss, g = M.loss_and_grad(w, X, T)
    idx = [0, 77, 511, 512, 600, 3000, 4671, 4672, 4736, 4800, 4864, 4865]
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (M.loss_and_grad(wp, X, T)[0] - M.loss_and_grad(wm, X, T)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_adam_hand_step():
    w = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    w1, m1, v1 = M.adam_step(w, g, np.zeros(2), np.zeros(2), 1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2, so w moves by lr * sign(g) (up to eps)
    assert np.allclose(w1, [0.9, -1.9], rtol=0, atol=1e-7)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_training_reduces_loss():
    w = M.init_weights(9)
    X = wl.normal(9, 4, 64 * 8).reshape(64, 8)
    T = np.stack([np.sin(X[:, 0]), X[:, 1] * 0.5], axis=1)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    l0 = M.loss_and_grad(w, X, T)[0]
    for t in range(1, 101):
        _, g = M.loss_and_grad(w, X, T)
        w, m, v = M.adam_step(w, g, m, v, t, lr=3e-3)
    assert M.loss_and_grad(w, X, T)[0] < 0.3 * l0
