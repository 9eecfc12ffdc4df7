"""The Heston workload of Sec. 4.1: the assembly against exact derivatives, and the oracle's
run at Tol = 1e-4 against the histories the paper prints in Figs. 2-3 (qualitative: the
trajectory of an adaptive controller changes with 1-ulp changes of A, so only its scale
can be compared)."""
import json
import os

import numpy as np

from oracle import phipm_oracle as O
from paper_0907_4631_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _heston_rhs(g, U, Us, Uss, Uv, Uvv, Usv, s, v):
    """The Heston operator applied to a smooth function (v > 0) or the v = 0 boundary operator."""
    inner = (0.5 * v * s * s * Uss + g.rho * g.lam * v * s * Usv + 0.5 * g.lam ** 2 * v * Uvv
             + (g.rd - g.rf) * s * Us + g.kappa * (g.eta - v) * Uv - g.rd * U)
    edge = (g.rd - g.rf) * s * Us + g.kappa * g.eta * Uv - g.rd * U
    return np.where(v == 0.0, edge, inner)


def test_heston_size():
    A, b0, b1, g = wl.heston_operator()
    assert A.n == 5100 == 100 * 51                 # Sec. 4.1: 5100 degrees of freedom
    # The printed differences give 44,900 nonzeros; the paper prints 44,800 (one fewer per
    # s-node, e.g. a two-point U_v at v = 0).  The assembly follows the printed formulas.
    assert A.nnz == 44900
    assert np.array_equal(b0, np.maximum(np.tile(g.s(), 51) - 100.0, 0.0))


def test_heston_assembly_exact_on_quadratics():
    """Second-order differences are exact on quadratics: away from the s = 0, s = S and v = V
    boundaries, (A U)_i equals the PDE operator (or the v = 0 boundary operator) at the node."""
    A, b0, b1, g = wl.heston_operator()
    s = np.tile(g.s(), g.nv)
    v = np.repeat(g.v(), g.ns)
    U = 0.3 * s * s + 2.0 * s * v - 5.0 * v * v + 7.0 * s - 11.0 * v + 13.0
    Us, Uss = 0.6 * s + 2.0 * v + 7.0, 0.6
    Uv, Uvv = 2.0 * s - 10.0 * v - 11.0, -10.0
    Usv = 2.0
    M = wl.csr_to_dense(A)
    AU = M @ U
    ref = _heston_rhs(g, U, Us, Uss, Uv, Uvv, Usv, s, v)
    i = np.tile(np.arange(g.ns), g.nv)
    j = np.repeat(np.arange(g.nv), g.ns)
    inner = (i >= 1) & (i <= g.ns - 2) & (j <= g.nv - 2)
    assert inner.sum() == 98 * 50
    assert np.allclose(AU[inner], ref[inner], rtol=1e-11, atol=1e-9 * np.abs(ref).max())


def test_heston_boundary_data_exact_for_u_equals_s():
    """U = s meets every boundary condition (U(0) = 0, U(s, V) = s, U_s(S) = 1) and, with
    r_f = 0, solves the PDE as a steady state: A U + b_1 = -r_f s = 0 at every node, which
    checks the Dirichlet data in b_1, the Neumann ghost and the v = 0 row together."""
    A, b0, b1, g = wl.heston_operator()
    U = np.tile(g.s(), g.nv)
    r = wl.csr_to_dense(A) @ U + b1
    assert np.abs(r).max() <= 1e-9 * np.abs(b1).max()


def test_heston_oracle_vs_figures_2_3():
    """Tol = 1e-4, T = 1.  The paper's run takes 132 steps on [0, 0.4] with tau ~ 3e-3 and
    accepted estimates ~ 2.5e-7 (medians of the printed data); the oracle's run has the same
    scale, meets the accept rule, and its result agrees with a Tol = 1e-9 run far below Tol."""
    with open(os.path.join(GOLDEN, "fig2_fig3_heston_tol1e-4.json")) as f:
        gold = json.load(f)
    pr = wl.heston_problem(tol=gold["tol"])
    trace = []
    u, st = O.phipm(gold["t_end"], pr.op, pr.b, pr.tol, 0, trace=trace)
    acc = [r for r in trace if r["accepted"]]
    early = [r for r in acc if r["t"] < 0.4]
    assert 0.6 * 132 <= len(early) <= 1.5 * 132
    tau_med = float(np.median([r["tau"] for r in early]))
    gold_tau = float(np.median([t for _, t in gold["tau_vs_t"]]))
    assert gold_tau / 2 <= tau_med <= 2 * gold_tau
    eps_med = float(np.median([r["eps"] for r in acc]))
    gold_eps = float(np.median([e for _, e in gold["error_estimate_vs_t"]]))
    assert gold_eps / 3 <= eps_med <= 3 * gold_eps
    assert all(r["omega"] <= 1.2 for r in acc)
    assert st.err_est_sum <= 1.2 * pr.tol
    u_fine, _ = O.phipm(gold["t_end"], pr.op, pr.b, 1e-9, 0)
    assert np.linalg.norm(u - u_fine) <= pr.tol


def test_heston_small_grid_vs_dense_augmented():
    """A 20 x 11 Heston grid (n = 220, the same assembly): the oracle's u(1) against the dense
    augmented exponential of Sidje's Theorem 1 (scipy's expm), within Tol (absolute, R6)."""
    A, b0, b1, g = wl.heston_operator(wl.HestonGrid(ns=20, nv=11))
    tol = 1e-6
    u, st = O.phipm(1.0, A, [b0, b1], tol, 0)
    from oracle import truth as T
    ut = T.solution_dense_augmented(wl.csr_to_dense(A), [b0, b1], 1.0)
    assert st.steps >= 5
    assert np.linalg.norm(u - ut) <= tol
