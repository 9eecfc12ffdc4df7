"""Exact answers for phipm problems, independent of the algorithm (Sec. 2).

TEST INFRASTRUCTURE ONLY (tests, smoke(), bench.py's CPU baseline).

  phi_scalar        phi_l(z) for scalars: Taylor series sum_k z^k/(k+l)! near 0,
                    else phi_0 = e^z and the recurrence of Eq. (phirelation),
                    phi_l = (phi_{l-1} - 1/(l-1)!)/z.
  phi_quadrature    the integral definition of Eq. (phifunctions) by
                    Gauss-Legendre quadrature (an independent route).
  solution_diagonal u_i = sum_k t^k phi_k(t lambda_i) b_{k,i} for diagonal A.
  solution_laplacian  Dirichlet Laplacian (1/2/3-D, scaled by 1/h^2) through its
                    orthonormal sine eigenbasis (DST-I as dense matrices).
  solution_dense_augmented  u = [I 0] exp(t [[A, W],[0, J]]) [b_0; e_p] with
                    W = [b_p .. b_1] and J the p x p upper shift: the dense
                    counterpart of Eq. (hathm) (Sidje 1998, Thm. 1), evaluated
                    with scipy.linalg.expm (not the oracle's Pade code).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg


def phi_scalar(ell: int, z):
    """phi_ell(z) for scalar or array z (real or complex)."""
    z = np.asarray(z, dtype=np.complex128 if np.iscomplexobj(z) else np.float64)
    out = np.empty_like(z)
    small = np.abs(z) < 1.0
    if np.any(small):
        zs = z[small]
        acc = np.zeros_like(zs)
        term = np.ones_like(zs) / math.factorial(ell)   # z^0/(0+ell)!
        for k in range(0, 40):
            acc = acc + term
            term = term * zs / (k + 1 + ell)
        out[small] = acc
    if np.any(~small):
        zb = z[~small]
        ph = np.exp(zb)
        for l in range(1, ell + 1):
            ph = (ph - 1.0 / math.factorial(l - 1)) / zb
        out[~small] = ph
    return out if out.ndim else out[()]


def phi_quadrature(ell: int, z, npts: int = 80):
    """Eq. (phifunctions) by Gauss-Legendre quadrature on [0, 1]."""
    if ell == 0:
        return np.exp(z)
    x, w = np.polynomial.legendre.leggauss(npts)
    th = 0.5 * (x + 1.0)
    w = 0.5 * w
    z = np.asarray(z)
    vals = np.exp(np.multiply.outer(z, 1.0 - th)) * th ** (ell - 1)
    return (vals @ w) / math.factorial(ell - 1)


def solution_diagonal(lams: np.ndarray, b: list, t: float) -> np.ndarray:
    u = np.zeros_like(np.asarray(b[0], dtype=np.float64))
    for k, bk in enumerate(b):
        u = u + (t ** k) * phi_scalar(k, t * lams) * bk
    return u


def dst_matrix(N: int) -> np.ndarray:
    """Orthonormal, symmetric DST-I matrix S[j,k] = sqrt(2/(N+1)) sin(pi (j+1)(k+1)/(N+1))."""
    j = np.arange(1, N + 1)
    return math.sqrt(2.0 / (N + 1)) * np.sin(np.pi * np.outer(j, j) / (N + 1))


def laplacian_eigenvalues(ndim: int, N: int) -> np.ndarray:
    """Eigenvalues of Delta_h on N^ndim interior points, as an array shaped (N,)*ndim
    in (z, y, x) order: lambda = -(4/h^2) sum_d sin^2(k_d pi h / 2)."""
    h = 1.0 / (N + 1)
    k = np.arange(1, N + 1)
    l1 = -(4.0 / h ** 2) * np.sin(k * np.pi * h / 2.0) ** 2
    lam = np.zeros((N,) * ndim)
    for d in range(ndim):
        shape = [1] * ndim
        shape[d] = N
        lam = lam + l1.reshape(shape)
    return lam


def _transform(X: np.ndarray, S: np.ndarray) -> np.ndarray:
    for ax in range(X.ndim):
        X = np.moveaxis(np.tensordot(S, X, axes=([1], [ax])), 0, ax)
    return X


def solution_laplacian(ndim: int, N: int, b: list, t: float) -> np.ndarray:
    S = dst_matrix(N)
    lam = laplacian_eigenvalues(ndim, N)
    u = np.zeros((N,) * ndim)
    for k, bk in enumerate(b):
        bh = _transform(np.asarray(bk, dtype=np.float64).reshape((N,) * ndim), S)
        u = u + (t ** k) * phi_scalar(k, t * lam) * bh
    return _transform(u, S).reshape(-1)


def solution_dense_augmented(A: np.ndarray, b: list, t: float) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    p = len(b) - 1
    At = np.zeros((n + p, n + p))
    At[:n, :n] = A
    for i in range(p):
        At[:n, n + i] = b[p - i]          # W = [b_p, ..., b_1]
        if i + 1 < p:
            At[n + i, n + i + 1] = 1.0    # J: upper shift
    z0 = np.zeros(n + p)
    z0[:n] = b[0]
    if p:
        z0[n + p - 1] = 1.0               # e_p
    return (scipy.linalg.expm(t * At) @ z0)[:n]
