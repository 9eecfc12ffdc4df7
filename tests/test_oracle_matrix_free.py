"""A matrix-free operator (R24): Sec. 3.5 accepts a function computing A b in place of A.
The oracle takes an object with apply(x) and the two scalars the method needs from A."""
import numpy as np

from oracle import phipm_oracle as O
from oracle import truth as T
from paper_0907_4631_gb300 import workloads as wl


class _MatrixFreeLaplacian:
    """The 2D Dirichlet Laplacian of workloads.laplacian(2, N) applied by slicing, with the
    two scalars a matrix-free operator supplies (R24)."""

    def __init__(self, N):
        self.N, self.n = N, N * N
        self.h2 = float((N + 1) ** 2)
        self.norm_inf = 8.0 * self.h2
        self.nnz = wl.laplacian(2, N).nnz()

    def apply(self, x):
        X = x.reshape(self.N, self.N)
        Y = -4.0 * X
        Y[1:, :] += X[:-1, :]
        Y[:-1, :] += X[1:, :]
        Y[:, 1:] += X[:, :-1]
        Y[:, :-1] += X[:, 1:]
        return (self.h2 * Y).reshape(-1)


def test_matrix_free_operator():
    """Sec. 3.5's implicit A: with symm = 1 the same Lanczos solve as the stencil operator;
    left undetected (symm = -1) it runs Arnoldi as a nonsymmetric A; both meet Tol against
    the sine expansion."""
    pr = wl.laplacian_2d_problem(N=12, p=2, t_end=0.01, tol=1e-8, seed=1012)
    mf = _MatrixFreeLaplacian(12)
    x = wl.normal(5, 1, mf.n)
    assert np.allclose(mf.apply(x), O.Operator(pr.op).matvec(x), rtol=1e-14, atol=1e-9)
    ut = T.solution_laplacian(2, 12, pr.b, pr.t_end)
    u_s, st_s = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1)
    u_f, st_f = O.phipm(pr.t_end, mf, pr.b, pr.tol, 1)
    assert np.linalg.norm(u_f - u_s) <= 1e-12 * np.linalg.norm(u_s)
    u_n, _ = O.phipm(pr.t_end, mf, pr.b, pr.tol, -1)
    for u in (u_f, u_n):
        assert np.linalg.norm(u - ut) <= 2.0 * pr.tol


# ---- the library's built-in matrix-free function (PHIPM_FN_VARCOEF_CONVDIFF) ----------
from oracle.matrix_free import VarCoefConvDiffOperator   # noqa: E402


def _dense(op):
    return np.column_stack([op.apply(np.eye(op.n)[:, j]) for j in range(op.n)])


def test_varcoef_with_constant_coefficients_is_the_pinned_stencil():
    """kappa = 1, no convection: the Dirichlet Laplacian; kappa = d, constant velocity: the
    convection-diffusion stencil of R14 (both pinned against the sine expansion and the
    assembly tests)."""
    N = 9
    data = wl.varcoef_convdiff(2, N, 0.0, seed=1)
    data.kappa = np.ones(N * N)
    x = wl.normal(11, 1, N * N)
    lap = O.Operator(wl.laplacian(2, N)).matvec(x)
    assert np.allclose(VarCoefConvDiffOperator(data).apply(x), lap, rtol=1e-13, atol=1e-9 * np.abs(lap).max())
    data.kappa = np.full(N * N, 2.5)
    data.vel = [np.full(N * N, 30.0), np.full(N * N, -12.0)]
    cd = O.Operator(wl.convection_diffusion_2d(N, 2.5, 30.0, -12.0)).matvec(x)
    assert np.allclose(VarCoefConvDiffOperator(data).apply(x), cd, rtol=1e-13, atol=1e-9 * np.abs(cd).max())
    data3 = wl.varcoef_convdiff(3, 5, 0.0, seed=2)
    data3.kappa = np.ones(125)
    y = wl.normal(12, 1, 125)
    assert np.allclose(VarCoefConvDiffOperator(data3).apply(y), O.Operator(wl.laplacian(3, 5)).matvec(y),
                       rtol=1e-13, atol=1e-9 * 36 * 8)


def test_varcoef_structure_and_norm():
    """Without convection the operator is symmetric and negative definite; norm_inf is the
    largest absolute row sum of the assembled matrix; with convection it is nonsymmetric."""
    for ndim, N in ((2, 7), (3, 4)):
        op = VarCoefConvDiffOperator(wl.varcoef_convdiff(ndim, N, 0.0, seed=3))
        D = _dense(op)
        assert np.allclose(D, D.T, rtol=0, atol=1e-12 * np.abs(D).max())
        assert np.linalg.eigvalsh(0.5 * (D + D.T)).max() < 0
        assert np.isclose(op.norm_inf, np.abs(D).sum(axis=1).max(), rtol=1e-13)
        opv = VarCoefConvDiffOperator(wl.varcoef_convdiff(ndim, N, 40.0, seed=3))
        Dv = _dense(opv)
        assert np.abs(Dv - Dv.T).max() > 1.0
        assert np.isclose(opv.norm_inf, np.abs(Dv).sum(axis=1).max(), rtol=1e-13)
        assert np.allclose(np.diag(Dv), np.diag(D))        # convection adds no diagonal


def test_varcoef_constant_kappa_meets_the_sine_expansion():
    """kappa = c constant, no convection: A = c Laplacian, so sum_k t^k phi_k(t c L) b_k =
    sum_k (c t)^k phi_k(c t L) (b_k / c^k), the sine expansion at time c t."""
    N, c = 10, 1.7
    data = wl.varcoef_convdiff(2, N, 0.0, seed=4)
    data.kappa = np.full(N * N, c)
    op = VarCoefConvDiffOperator(data)
    b = [wl.normal(13, k, N * N) for k in range(3)]
    t, tol = 0.01, 1e-9
    u, _ = O.phipm(t, op, b, tol, 1)
    ut = T.solution_laplacian(2, N, [bk / c ** k for k, bk in enumerate(b)], c * t)
    assert np.linalg.norm(u - ut) <= 2.0 * tol
