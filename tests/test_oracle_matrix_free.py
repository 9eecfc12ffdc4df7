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
