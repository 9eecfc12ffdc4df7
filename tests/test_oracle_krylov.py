"""Pins of the oracle's Krylov projections (Algorithms 1, 2) and one attempt
(Eqs. phipapprox, errest, phipapprox2) against dense truths."""
import numpy as np
import pytest
import scipy.linalg

from oracle import phipm_oracle as O
from oracle import truth as T
from paper_0907_4631_gb300 import workloads as wl


def _dense(A):
    return wl.csr_to_dense(A) if hasattr(A, "rowptr") else wl.csr_to_dense(wl.stencil_to_csr(A))


def test_arnoldi_relation_and_orthonormality():
    A = wl.convection_diffusion_2d(10, 1.0, 30.0, -20.0)
    op = O.Operator(A)
    v = wl.normal(3, 0, op.n)
    m = 25
    V, H, me = O.arnoldi(op.matvec, v, m, 0.0)
    assert me == m
    D = _dense(A)
    assert np.allclose(np.tril(H, -2), 0.0)
    resid = D @ V[:m].T - V.T @ H
    assert np.linalg.norm(resid) <= 1e-12 * np.linalg.norm(D, 2)
    assert np.linalg.norm(V @ V.T - np.eye(m + 1)) <= 1e-7   # MGS: loss ~ eps * cond(K)
    assert np.allclose(V[:m] @ D @ V[:m].T, H[:m], atol=1e-7 * np.linalg.norm(D, 2))
    assert np.allclose(V[0], v / np.linalg.norm(v))


def test_lanczos_matches_arnoldi_on_symmetric():
    A = wl.laplacian(2, 12)
    op = O.Operator(A)
    v = wl.normal(5, 0, op.n)
    m = 20
    Va, Ha, _ = O.arnoldi(op.matvec, v, m, 0.0)
    Vl, Tl, _ = O.lanczos(op.matvec, v, m, 0.0)
    scale = op.norm_inf()
    assert np.allclose(Tl[:m], Tl[:m].T, atol=0)
    assert np.allclose(np.triu(Tl, 2), 0) and np.allclose(np.tril(Tl, -2), 0)
    assert np.allclose(Tl, Ha, atol=1e-9 * scale)
    assert np.allclose(Vl, Va, atol=1e-7)


def test_breakdown_gives_exact_result():
    D = np.diag([-1.0, -2.0, -5.0, -9.0, -0.5, -3.0])
    A = wl.dense_to_csr(D)
    op = O.Operator(A)
    v = np.ones(6)
    V, H, me = O.arnoldi(op.matvec, v, 10, 1e-12 * op.norm_inf())
    assert me == 6 and H[me, me - 1] == 0.0
    for p in [0, 1, 3]:
        F, eps, me2, _, beta = O.krylov_attempt(op.matvec, O.arnoldi, v, 0.7, 10, p, 1e-12 * op.norm_inf())
        ref = 0.7 ** p * T.phi_scalar(p, 0.7 * np.diag(D)) * v
        assert eps == 0.0 and me2 == 6
        assert np.allclose(F, ref, rtol=1e-12, atol=1e-14)


def _exact_phi_action(D, tau, p, v):
    lam, X = np.linalg.eig(tau * D)
    return (tau ** p) * (X @ (T.phi_scalar(p, lam) * np.linalg.solve(X, v))).real


@pytest.mark.parametrize("p", [0, 1, 2, 4])
@pytest.mark.parametrize("tau,m", [(3e-3, 5), (5e-3, 8)])
def test_corrector_and_error_estimate(p, tau, m):
    """Eq. (errorseries): the corrector is the leading error term, so the corrected F
    beats the uncorrected one, and eps measures the uncorrected error (reading R4).
    Truth: tau^p phi_p(tau A) v from the dense augmented exponential (scipy)."""
    A = wl.convection_diffusion_2d(12, 1.0, 20.0, 10.0)
    op = O.Operator(A)
    D = _dense(A)
    v = wl.normal(9, p, op.n)
    F, eps, me, _, beta = O.krylov_attempt(op.matvec, O.arnoldi, v, tau, m, p, 0.0)
    ref = T.solution_dense_augmented(D, [np.zeros(op.n)] * p + [v], tau)
    V, H, _ = O.arnoldi(op.matvec, v, m, 0.0)
    E = O.expm_pade13(O.augmented_matrix(H[:m, :m], tau, p))
    phi_p = E[:m, m + p - 1] if p else E[:m, 0]
    F_plain = tau ** p * beta * V[:m].T @ phi_p           # Eq. (phipapprox) alone
    err_plain = np.linalg.norm(F_plain - ref)
    err_corr = np.linalg.norm(F - ref)
    assert err_corr < 0.6 * err_plain
    assert 0.5 * err_plain < eps < 3.0 * err_plain


def test_krylov_approximation_converges_to_dense():
    A = wl.random_sparse(21, 40, 4, 2.0)
    op = O.Operator(A)
    D = _dense(A)
    v = wl.normal(21, 7, 40)
    for p in [0, 2]:
        F, eps, me, _, _ = O.krylov_attempt(op.matvec, O.arnoldi, v, 0.5, 40, p, 1e-12 * op.norm_inf())
        assert np.allclose(F, _exact_phi_action(D, 0.5, p, v), rtol=1e-10, atol=1e-11)
