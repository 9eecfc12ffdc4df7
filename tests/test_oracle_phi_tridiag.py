"""phi of the symmetric Lanczos matrix computed directly (the alternative Sec. 5 proposes
to the augmented exponential): the scalar phi functions against their integral
definition, the tridiagonal route against the oracle's augmented Pade route, and the
whole method with it against the Laplacian's sine expansion."""
import numpy as np
import pytest

from oracle import phipm_oracle as O
from oracle import truth as T
from paper_0907_4631_gb300 import workloads as wl


def test_phi_scalars_against_the_integral_definition():
    z = np.array([-60.0, -7.5, -1.0, -0.999, -0.3, 0.0, 1e-9, 0.7, 1.0, 3.0])
    ph = O.phi_scalars(z, 5)
    assert np.allclose(ph[0], np.exp(z), rtol=1e-15, atol=0)
    for k in range(1, 6):
        ref = T.phi_quadrature(k, z)
        assert np.allclose(ph[k], ref, rtol=1e-12, atol=1e-300), k


def _random_tridiagonal(seed, m, scale):
    d = -scale * wl.uniform(seed, 1, m, 0.0, 1.0)
    e = scale * 0.5 * wl.uniform(seed, 2, m - 1, -1.0, 1.0)
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


@pytest.mark.parametrize("m,p,scale", [(1, 0, 1.0), (6, 1, 0.5), (12, 3, 4.0), (30, 4, 40.0), (20, 2, 300.0)])
def test_tridiagonal_route_equals_augmented_exponential(m, p, scale):
    Tm = _random_tridiagonal(100 + m, m, scale)
    tau = 0.37
    a, b = O.phi_columns_tridiagonal(Tm, tau, p)
    E = O.expm_pade13(O.augmented_matrix(Tm, tau, p))
    ea = E[:m, m + p - 1] if p >= 1 else E[:m, 0]
    eb = E[:m, m + p]
    assert np.linalg.norm(a - ea) <= 1e-12 * max(1.0, np.linalg.norm(ea))
    assert np.linalg.norm(b - eb) <= 1e-12 * max(1.0, np.linalg.norm(eb))


def test_phipm_with_the_tridiagonal_route():
    """The full method on the 2D Laplacian (Lanczos) with phi taken through the eigen-
    decomposition: within Tol of the sine expansion, and equal to the augmented route's
    result up to rounding (the controller, and so the trajectory, is the same)."""
    pr = wl.laplacian_2d_problem(N=16, p=3, t_end=0.01, tol=1e-8, seed=1016)
    u_e, st_e = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1, params=dict(phi_method="eigen"))
    u_a, st_a = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1)
    ut = T.solution_laplacian(2, 16, pr.b, pr.t_end)
    assert np.linalg.norm(u_e - ut) <= 2.0 * pr.tol
    assert np.linalg.norm(u_e - u_a) <= 1e-10 * np.linalg.norm(u_a)
    assert (st_e.steps, st_e.rejects) == (st_a.steps, st_a.rejects)


def test_planted_transposed_eigenvectors(monkeypatch):
    """Q^T in place of Q in the tridiagonal route must fail the comparison above."""
    def bad(T_m, tau, p):
        lam, Q = np.linalg.eigh(T_m)
        ph = O.phi_scalars(tau * lam, p + 1)
        return Q.T @ (ph[p] * Q[0, :]), Q.T @ (ph[p + 1] * Q[0, :])
    monkeypatch.setattr(O, "phi_columns_tridiagonal", bad)
    with pytest.raises(AssertionError):
        test_tridiagonal_route_equals_augmented_exponential(12, 3, 4.0)

