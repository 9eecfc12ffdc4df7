"""Pins of the fixed-dimension variant phip and of the Sec. 4.2 nine-point workloads.

  * the nine-point matrix: the size the paper prints (n = 900, nnz = 7,744) and its
    eigenvalues from the closed form of a separable stencil;
  * the round trip e^{-tA} e^{tA} b_0 = b_0 (exact in exact arithmetic; Experiment 1);
  * phip keeps m and adapts only tau, and still meets the tolerance against the
    sine eigen-expansion of the Laplacian;
  * phip against the dense augmented exponential on the Experiment 2 stand-in."""
import math

import numpy as np
import pytest

from oracle import phipm_oracle as O
from oracle import truth as T
from paper_0907_4631_gb300 import workloads as wl


def test_nine_point_matrix_size_and_spectrum():
    S = wl.nine_point(30)
    assert (S.n, S.nnz) == (900, 7744)             # Sec. 4.2: order 900, 7,744 nonzeros
    D = wl.csr_to_dense(S)
    assert np.array_equal(D, D.T)
    # S = 9 I - (T (x) T) with T = tridiag(1, 1, 1): eigenvalues 9 - (1 + 2 cos a)(1 + 2 cos b),
    # a, b = k pi / 31, k = 1..30
    c = 1.0 + 2.0 * np.cos(np.arange(1, 31) * math.pi / 31)
    lam = np.sort((9.0 - np.outer(c, c)).ravel())
    assert np.allclose(np.linalg.eigvalsh(D), lam, rtol=0, atol=1e-12)
    assert 0.0 < lam[0] and lam[-1] < 12.0


@pytest.mark.parametrize("adapt_m", [True, False])
def test_round_trip_returns_b0(adapt_m):
    """Experiment 1 (third case): w = e^{tA} b_0 at Tol = 1e-14, then e^{-tA} w.  The reverse
    pass amplifies the forward pass's absolute error in the top eigenmode by up to
    e^{t lambda_max} = e^{2 * 12}, so the bound is 1e-5 relative (the paper reports
    3.9e-6 for phipm and 1.8e-6 for phip on its matrix)."""
    A, B, b0, t, tol = wl.nine_point_round_trip()
    prm = None if adapt_m else dict(adapt_m=False, m_init=30)
    w, _ = O.phipm(t, A, [b0], tol, 1, params=prm)
    r, _ = O.phipm(t, B, [w], tol, 1, params=prm)
    assert np.linalg.norm(r - b0) / np.linalg.norm(b0) <= 1e-5
    # the forward result itself against the closed form through the eigen-decomposition
    lam, Q = np.linalg.eigh(wl.csr_to_dense(A))
    w_exact = Q @ (np.exp(t * lam) * (Q.T @ b0))
    assert np.linalg.norm(w - w_exact) <= 10 * tol + 1e-13 * np.linalg.norm(w_exact)


@pytest.mark.parametrize("m", [6, 12])
def test_phip_keeps_m_and_meets_tol(m):
    """phip on the 2D Laplacian: every attempt uses the same m, every attempt takes the
    tau branch, tau stays within Algorithm 3's factors, and u meets Tol."""
    pr = wl.laplacian_2d_problem(N=16, p=2, t_end=0.02, tol=1e-8, seed=1016)
    trace = []
    u, st = O.phip(pr.t_end, pr.op, pr.b, pr.tol, 1, m=m, trace=trace)
    assert st.steps >= 2
    assert all(r["m"] == m and r["next_m"] == m for r in trace)
    assert all(r["branch"] == "tau" for r in trace)
    for r in trace:
        assert r["tau"] / 5 * (1 - 1e-15) <= r["next_tau"] <= 2 * r["tau"] * (1 + 1e-15)
    ut = T.solution_laplacian(2, 16, pr.b, pr.t_end)
    assert np.linalg.norm(u - ut) <= 2.0 * pr.tol


def test_phip_rejects_then_shrinks_tau():
    """A small fixed m forces rejections; each rejected attempt is retried with a smaller tau
    (m cannot change), and the step that follows is accepted at omega <= delta."""
    pr = wl.laplacian_2d_problem(N=16, p=1, t_end=0.05, tol=1e-10, seed=1017)
    trace = []
    u, st = O.phip(pr.t_end, pr.op, pr.b, pr.tol, 1, m=5, trace=trace)
    assert st.rejects >= 1
    for a, c in zip(trace, trace[1:]):
        if not a["accepted"]:
            assert c["tau"] < a["tau"] and c["m"] == a["m"] == 5
    assert all(r["omega"] <= 1.2 for r in trace if r["accepted"])
    ut = T.solution_laplacian(2, 16, pr.b, pr.t_end)
    assert np.linalg.norm(u - ut) <= 2.0 * pr.tol


@pytest.mark.parametrize("adapt_m", [True, False])
def test_nine_point_phi_sum_vs_dense_augmented(adapt_m):
    """Experiment 2 stand-in: sum_{k<=4} t^k phi_k(tA) 1 with t = 2, Tol = 2^-26, by phipm and by
    phip (m = 30), against the dense augmented exponential (scipy's expm, Sidje's Thm. 1)."""
    pr = wl.nine_point_phi_sum_problem()
    fn = O.phipm if adapt_m else O.phip
    u, st = fn(pr.t_end, pr.op, pr.b, pr.tol, 1)
    ut = T.solution_dense_augmented(wl.csr_to_dense(pr.op), pr.b, pr.t_end)
    assert np.linalg.norm(u - ut) <= 2.0 * pr.tol
