"""Pins of the oracle's scalar phi functions, Pade exponential and augmented matrix.

Checked against what Sec. 2-3.1 fix: the closed forms of phi_1..phi_3, the
recurrence of Eq. (phirelation), the integral definition of Eq. (phifunctions),
textbook exponentials (2x2 triangular, nilpotent, rotation, diagonal),
exp(A) exp(-A) = I, scipy's independent expm, and the augmented-matrix identity
of Eq. (hathm) via an eigen-decomposition route."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import phipm_oracle as O
from oracle import truth as T

ZS = [-87.0, -20.0, -3.5, -1.0, -0.7, -1e-3, 1e-6, 0.3, 0.999, 1.0, 2.5, 10.0]


@pytest.mark.parametrize("z", ZS)
def test_phi_closed_forms(z):
    ez = math.exp(z)
    closed = {
        1: (ez - 1) / z,
        2: (ez - 1 - z) / z ** 2,
        3: (ez - 1 - z - z * z / 2) / z ** 3,
    }
    for ell, ref in closed.items():
        if abs(z) < 1e-2:     # the closed forms cancel catastrophically near 0
            ref = sum(z ** k / math.factorial(k + ell) for k in range(30))
        assert T.phi_scalar(ell, z) == pytest.approx(ref, rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("z", ZS)
def test_phi_recurrence_and_integral(z):
    for ell in range(0, 6):
        lhs = T.phi_scalar(ell, z)
        if ell >= 1:
            rhs = z * T.phi_scalar(ell + 1, z) + 1.0 / math.factorial(ell)
            assert lhs == pytest.approx(rhs, rel=1e-11, abs=1e-14)
        if abs(z) <= 20:
            assert lhs == pytest.approx(T.phi_quadrature(ell, z), rel=1e-11, abs=1e-300)


def test_phi_at_zero_and_complex():
    for ell in range(6):
        assert T.phi_scalar(ell, 0.0) == pytest.approx(1.0 / math.factorial(ell), rel=1e-15)
    z = 2.0 + 3.0j
    assert T.phi_scalar(1, z) == pytest.approx((np.exp(z) - 1) / z, rel=1e-13)


def test_pade13_coefficients():
    c = O.pade13_coefficients()
    assert c[0] == 1.0 and c[1] == pytest.approx(0.5, rel=1e-15)
    for j in range(13):
        assert c[j + 1] / c[j] == pytest.approx((13 - j) / ((26 - j) * (j + 1)), rel=1e-14)
    # the scalar approximant reaches double precision inside |x| <= theta_13
    for x in [-5.37, -1.0, 0.25, 3.0, 5.37]:
        P = sum(cj * x ** j for j, cj in enumerate(c))
        Q = sum(cj * (-x) ** j for j, cj in enumerate(c))
        assert P / Q == pytest.approx(math.exp(x), rel=5e-15)


def test_squarings_and_cost_factor():
    assert O.squarings(0.0, 5.37) == 0
    assert O.squarings(5.37, 5.37) == 0
    assert O.squarings(5.3701, 5.37) == 1
    assert O.squarings(10.74, 5.37) == 1
    assert O.squarings(10.7401, 5.37) == 2
    assert O.expm_cost_factor(40.0) == pytest.approx(44.0 / 3.0 + 2 * 3)


def test_expm_textbook_cases():
    a, b, c = -3.0, 7.0, 0.5
    E = O.expm_pade13(np.array([[a, b], [0.0, c]]))
    ref = np.array([[math.exp(a), b * (math.exp(a) - math.exp(c)) / (a - c)], [0.0, math.exp(c)]])
    assert np.allclose(E, ref, rtol=1e-13, atol=1e-15)
    th = 40.0
    E = O.expm_pade13(np.array([[0.0, -th], [th, 0.0]]))
    assert np.allclose(E, [[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]], atol=1e-12)
    J = np.diag(np.ones(5), 1)
    E = O.expm_pade13(J)
    ref = sum(np.linalg.matrix_power(J, k) / math.factorial(k) for k in range(6))
    assert np.allclose(E, ref, rtol=1e-14, atol=1e-15)
    d = np.array([-30.0, -1.0, 0.0, 2.0])
    assert np.allclose(O.expm_pade13(np.diag(d)), np.diag(np.exp(d)), rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("scale", [0.01, 1.0, 7.0, 45.0, 300.0])
def test_expm_vs_scipy_and_inverse(scale):
    rng = np.random.default_rng(7)
    A = np.triu(rng.standard_normal((30, 30)), -1)       # Hessenberg, like H_hat
    A *= scale / np.abs(A).sum(axis=0).max()
    A -= np.diag(np.full(30, scale / 3))                  # decaying, like tau*H
    E = O.expm_pade13(A)
    R = scipy.linalg.expm(A)
    assert np.linalg.norm(E - R, 1) <= 1e-12 * max(1.0, np.linalg.norm(R, 1)) * max(1.0, scale)
    if scale <= 45:
        Ei = O.expm_pade13(-A)
        assert np.linalg.norm(E @ Ei - np.eye(30), 1) <= 1e-10 * max(1.0, scale) ** 2


@pytest.mark.parametrize("p", [0, 1, 2, 4])
def test_augmented_matrix_identity(p):
    """Top m entries of column m+j-1 of exp(H_hat) equal phi_j(tau H) e_1 (Eq. hathm, R2)."""
    rng = np.random.default_rng(11 + p)
    m, tau = 12, 0.37
    H = np.triu(rng.standard_normal((m, m)), -1) * 3.0 - 4.0 * np.eye(m)
    Hh = O.augmented_matrix(H, tau, p)
    assert Hh.shape == (m + p + 1, m + p + 1)
    E = O.expm_pade13(Hh)
    lam, X = np.linalg.eig(tau * H)
    Xi_e1 = np.linalg.solve(X, np.eye(m)[:, 0])
    for j in range(0, p + 2):
        ref = (X @ (T.phi_scalar(j, lam) * Xi_e1)).real
        col = 0 if j == 0 else m + j - 1
        assert np.allclose(E[:m, col], ref, rtol=1e-10, atol=1e-12), j
