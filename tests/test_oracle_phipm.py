"""Pins of the full oracle (Algorithm 3) against truths fixed by the mathematics.

  * Dirichlet Laplacian (2D/3D) through its sine eigen-expansion;
  * diagonal A through the scalar phi functions (Sec. 2);
  * nonsymmetric sparse A through the dense augmented exponential (scipy);
  * Lemma 2.1: restarting at t1 with shifted inputs gives the same answer;
  * invariants of the accept rule (omega <= delta), of the time grid, and
    hand-computed controller values (Eqs. 2, 3, 4, 5, 6, 7, tau_0)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import phipm_oracle as O
from oracle import truth as T
from paper_0907_4631_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N,p,tol", [(8, 3, 1e-8), (16, 3, 1e-8), (32, 3, 1e-8), (16, 1, 1e-5), (12, 0, 1e-10)])
def test_laplacian_2d_vs_sine_expansion(N, p, tol):
    pr = wl.laplacian_2d_problem(N=N, p=p, t_end=0.01, tol=tol, seed=1000 + N)
    trace = []
    u, st = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1, trace=trace)
    ut = T.solution_laplacian(2, N, pr.b, pr.t_end)
    assert np.linalg.norm(u - ut) <= 2.0 * tol
    assert st.steps >= 1 and st.expms == len(trace)


def test_c1_configuration_vs_sine_expansion():
    """Plain phipm FP64 configuration: 32x32 Laplacian, p=3, t=0.01, tol=1e-8."""
    pr = wl.laplacian_2d_problem()
    u, st = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, -1)
    ut = T.solution_laplacian(2, 32, pr.b, pr.t_end)
    assert np.linalg.norm(u - ut) / np.linalg.norm(ut) <= 1e-8


@pytest.mark.parametrize("N,tol", [(6, 1e-8), (10, 1e-5)])
def test_laplacian_3d_vs_sine_expansion(N, tol):
    pr = wl.laplacian_3d_problem(N=N, p=2, t_end=1e-2, tol=tol, seed=3000 + N, precision="f64")
    u, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1)
    ut = T.solution_laplacian(3, N, pr.b, pr.t_end)
    assert np.linalg.norm(u - ut) <= 2.0 * tol


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_diagonal_vs_scalar_phi(p):
    n = 50
    lam = -np.geomspace(1e-2, 3e3, n)
    A = wl.dense_to_csr(np.diag(lam))
    b = [wl.normal(77, k, n) for k in range(p + 1)]
    u, _ = O.phipm(1.0, A, b, 1e-9, 1)
    ut = T.solution_diagonal(lam, b, 1.0)
    assert np.linalg.norm(u - ut) <= 2e-9


@pytest.mark.parametrize("p", [0, 1, 2, 4])
@pytest.mark.parametrize("seed", [1, 2])
def test_nonsymmetric_vs_dense_augmented(p, seed):
    A = wl.random_sparse(seed, 40, 5, 3.0)
    b = [wl.normal(seed, 10 + k, 40) for k in range(p + 1)]
    u, st = O.phipm(2.0, A, b, 1e-10, -1)
    ut = T.solution_dense_augmented(wl.csr_to_dense(A), b, 2.0)
    assert np.linalg.norm(u - ut) <= 5e-10


def test_convection_diffusion_vs_dense_augmented():
    pr = wl.convdiff_2d_problem(N=14, p=4, t_end=1e-3, tol=1e-8, seed=2014)
    u, st = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, -1)
    ut = T.solution_dense_augmented(wl.csr_to_dense(pr.op), pr.b, pr.t_end)
    assert np.linalg.norm(u - ut) <= 2e-8
    assert st.steps >= 1


def test_lemma_2_1_restart():
    """Solving to t1 and restarting with b'_0 = u(t1), b'_i = sum_l t1^l/l! b_{i+l}
    (Lemma 2.1, Eq. steppre) agrees with one solve to t_end."""
    pr = wl.convdiff_2d_problem(N=16, p=3, t_end=2e-3, tol=1e-10, seed=2016)
    u_full, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    t1 = 0.7e-3
    u1, _ = O.phipm(t1, pr.op, pr.b, pr.tol, 0)
    b2 = O.shifted_inputs(pr.b, t1)
    b2[0] = u1
    u2, _ = O.phipm(pr.t_end - t1, pr.op, b2, pr.tol, 0)
    ut = T.solution_dense_augmented(wl.csr_to_dense(pr.op), pr.b, pr.t_end)
    assert np.linalg.norm(u2 - ut) <= 1e-9
    assert np.linalg.norm(u_full - ut) <= 1e-9


def test_accept_rule_and_time_grid_invariants():
    pr = wl.convdiff_2d_problem(N=20, p=2, t_end=1e-3, tol=1e-7, seed=2020)
    trace = []
    u, st = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0, trace=trace)
    acc = [r for r in trace if r["accepted"]]
    assert len(acc) == st.steps and len(trace) - len(acc) == st.rejects
    for r in acc:       # omega <= delta  <=>  eps <= delta tau Tol / t_end
        assert r["eps"] <= 1.2 * r["tau"] * pr.tol / pr.t_end * (1 + 1e-12)
    for r in trace:
        if not r["accepted"]:
            assert r["omega"] > 1.2
    assert sum(r["tau"] for r in acc) == pytest.approx(pr.t_end, rel=1e-14)
    ts = [r["t"] for r in acc]
    assert all(b > a for a, b in zip(ts, ts[1:]))
    for a, b in zip(trace, trace[1:]):          # clamps of Algorithm 3
        if b["m"] == a["next_m"]:
            assert (3 * a["m"]) // 4 <= b["m"] <= math.ceil(4 * a["m"] / 3)
        assert b["tau"] <= 2 * a["tau"] * (1 + 1e-15)


def test_edge_cases():
    A = wl.laplacian(2, 6)
    n = A.n
    z = np.zeros(n)
    u, st = O.phipm(1e-2, A, [z, z, z], 1e-8, 1)            # every b_k = 0
    assert np.all(u == 0) and st.steps == 0
    b1 = wl.normal(4, 1, n)
    u, _ = O.phipm(1e-2, A, [z, b1], 1e-10, 1)               # b_0 = 0
    assert np.allclose(u, T.solution_laplacian(2, 6, [z, b1], 1e-2), atol=1e-10)
    Z = wl.dense_to_csr(np.zeros((5, 5)))                    # A = 0
    b = [wl.normal(4, k, 5) for k in range(4)]
    u, _ = O.phipm(0.3, Z, b, 1e-8, -1)
    assert np.allclose(u, sum(0.3 ** k / math.factorial(k) * bk for k, bk in enumerate(b)), rtol=1e-14)
    small = wl.random_sparse(3, 5, 3, 1.0)                    # n < m: happy breakdown
    b = [wl.normal(5, k, 5) for k in range(3)]
    u, st = O.phipm(1.0, small, b, 1e-12, -1)
    assert np.allclose(u, T.solution_dense_augmented(wl.csr_to_dense(small), b, 1.0), rtol=1e-11, atol=1e-12)
    u_def, _ = O.phipm(1e-2, A, [b1], 0.0, 1)                 # tol <= 0 -> default 1e-7
    u_7, _ = O.phipm(1e-2, A, [b1], 1e-7, 1)
    assert np.array_equal(u_def, u_7)


def test_initial_step_formula():
    """Eq. (tau_0) evaluated directly (no logarithms) for moderate values."""
    for nA, nb, tol, mbar in [(1.0, 1.0, 1e-7, 37.0), (2.1e6, 4.5, 1e-8, 37.0), (50.0, 0.3, 1e-4, 20.0)]:
        direct = 10.0 / nA * (tol * ((mbar + 1) / math.e) ** (mbar + 1) * math.sqrt(2 * math.pi * (mbar + 1))
                              / (4 * nA * nb)) ** (1.0 / mbar)
        assert O.initial_tau(nA, nb, tol, mbar) == pytest.approx(direct, rel=1e-12)
    assert O.initial_tau(1.0, 1.0, 1e-7, 37.0) == pytest.approx(100.72, rel=1e-4)


def test_controller_hand_cases():
    prm = dict(O.DEFAULTS)
    # fresh attempt: q = m/4 = 5, kappa = 2 (Alg. 4 default branches)
    mem = O.AttemptMemory()
    q, tn, k, mn = O.controller(1e-6, 10.0, 1e-3, 20, mem, prm)
    assert q == 5.0 and k == 2.0
    assert tn == pytest.approx(6.56420e-4, rel=1e-5)           # 1e-3 * 0.08^(1/6)
    assert mn == pytest.approx(23.643856, rel=1e-7)            # 20 + log2(12.5)
    # previous attempt rejected after a tau change: Eq. (6) as read in R7
    mem = O.AttemptMemory(rejected=True, tau_changed=True, eps_old=1e-6, tau_old=1e-3, m_old=20)
    q, tn, k, mn = O.controller(1e-8, 0.2, 5e-4, 20, mem, prm)
    assert q == pytest.approx(5.643856, rel=1e-6)              # log2(100) - 1
    assert tn == pytest.approx(5e-4 * 4.0 ** (1 / 6.643856), rel=1e-6)
    assert k == 2.0 and mn == pytest.approx(18.0, rel=1e-12)
    # previous attempt rejected after an m change: Eq. (7)
    mem = O.AttemptMemory(rejected=True, m_changed=True, eps_old=1e-6, tau_old=1e-3, m_old=20)
    q, tn, k, mn = O.controller(1e-8, 0.1, 1e-3, 24, mem, prm)
    assert q == 6.0 and k == pytest.approx(10 ** 0.5, rel=1e-12)
    assert mn == pytest.approx(24 - 1.80618, rel=1e-5)
    # kept values (Alg. 4 second branches)
    mem = O.AttemptMemory(rejected=True, m_changed=True, q_from_formula=True, q_hat=3.3,
                          eps_old=1e-6, tau_old=1e-3, m_old=20)
    q, *_ = O.controller(1e-7, 1.5, 1e-3, 24, mem, prm)
    assert q == 3.3
    # eps = 0: tau_new = inf, m_new = -inf (reading R13)
    q, tn, k, mn = O.controller(0.0, 0.0, 1e-3, 20, O.AttemptMemory(), prm)
    assert tn == math.inf and mn == -math.inf


def test_cost_model_hand_values():
    M = 44.0 / 3.0
    assert O.step_cost(10, 2, 100, 20, M, False) == pytest.approx(1200 + 108 * 20 + M * 13 ** 3)
    assert O.step_cost(10, 2, 100, 20, M, True) == pytest.approx(1200 + 3 * 12 * 20 + M * 13 ** 3)
    assert O.total_cost(0.3, 10, 1.0, 2, 100, 20, M, True) == pytest.approx(4 * O.step_cost(10, 2, 100, 20, M, True))
    assert O.total_cost(math.inf, 10, 1.0, 2, 100, 20, M, True) == 0.0


def test_paper_constants_are_the_oracles():
    c = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    d = O.DEFAULTS
    assert d["gamma"] == c["gamma"] and d["delta"] == c["delta"] and d["m_init"] == c["m_init"]
    assert d["theta13"] == c["theta13"]
    assert O.expm_cost_factor(0.0) == pytest.approx(c["M_const"])
    assert O.expm_cost_factor(4 * 5.37) - O.expm_cost_factor(0.0) == pytest.approx(2 * c["M_per_squaring"])


def test_paper_fig2_fig3_data_obey_the_readings():
    """The paper's printed Heston histories (Sec. 4.1, Figs. 2-3, Tol 1e-4, t_end 1):
    t advances by the plotted tau (R9); each accepted estimate satisfies
    omega = t_end eps/(tau Tol) <= delta (R4, R10) with omega clustered near gamma;
    m and tau move within Algorithm 3's clamps."""
    g = json.load(open(os.path.join(GOLDEN, "fig2_fig3_heston_tol1e-4.json")))
    tol, t_end = g["tol"], g["t_end"]
    tgrid = [t for t, _ in g["error_estimate_vs_t"]]
    taus = dict((round(t, 6), tau) for t, tau in g["tau_vs_t"])
    taus[0.0] = tgrid[1] - tgrid[0]
    omegas = []
    for k, (t, eps) in enumerate(g["error_estimate_vs_t"]):
        tau = taus[round(t, 6)]
        if k + 1 < len(tgrid):
            assert tgrid[k + 1] == pytest.approx(t + tau, rel=2e-5)
        omegas.append(t_end * eps / (tau * tol))
    assert max(omegas) <= 1.2 * (1 + 1e-4)
    assert 0.6 <= float(np.median(omegas)) <= 1.0
    ms = [m for _, m in g["m_vs_t"]]
    for a, b in zip(ms, ms[1:]):
        assert math.floor(0.75 * a) <= b <= math.ceil(4 * a / 3)
    tv = [tau for _, tau in g["tau_vs_t"]]
    for a, b in zip(tv, tv[1:]):
        assert a / 5 <= b <= 2 * a


def test_long_horizon_error_budget():
    """With omega = t_end eps/(tau Tol) the accepted estimates sum to at most
    delta*Tol over the whole horizon, so the global error stays near Tol even
    for t_end >> 1 (the factor t_end makes the method invariant under time scaling)."""
    n = 40
    lam = -np.geomspace(1e-3, 30.0, n)
    A = wl.dense_to_csr(np.diag(lam))
    b = [wl.normal(91, k, n) for k in range(2)]
    tol = 1e-8
    u, st = O.phipm(50.0, A, b, tol, 1)
    assert st.steps >= 3
    assert st.err_est_sum <= 1.2 * tol * (1 + 1e-12)
    assert np.linalg.norm(u - T.solution_diagonal(lam, b, 50.0)) <= 3 * tol


def test_m_branch_at_m_max_changes_tau():
    """Reading R19: at m = m_max with the tolerance missed, the cost comparison can favour the
    m branch although m cannot grow; tau must change instead, and the result stays accurate
    (dense augmented exponential).  A strongly convective problem with m_max = 24 meets it."""
    st = wl.convection_diffusion_2d(16, 1.0, 800.0, 240.0)
    op = wl.stencil_to_csr(st)
    b = [wl.normal(11, k, st.n) for k in range(2)]
    trace = []
    u, stats = O.phipm(4e-3, op, b, 1e-8, 0, params=dict(m_max=24), trace=trace)
    blocked = [r for r in trace if r["m"] == 24 and not r["accepted"] and r["cost_m"] <= r["cost_tau"]]
    assert blocked, "the case no longer reaches the m bound"
    for r in blocked:
        assert r["branch"] == "tau" and r["next_tau"] < r["tau"]
    # consecutive attempts never repeat the same (tau, m)
    for a, c in zip(trace, trace[1:]):
        if not a["accepted"]:
            assert (a["tau"], a["m"]) != (c["tau"], c["m"])
    ut = T.solution_dense_augmented(wl.csr_to_dense(op), b, 4e-3)
    assert np.linalg.norm(u - ut) <= 2e-8
