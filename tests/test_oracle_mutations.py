"""Planted mistakes: each plausible slip in the oracle must make at least one pin fail.

Every mistake is planted in the oracle, on the CPU, through monkeypatch, and
the pin that should catch it is run expecting an AssertionError."""
import math

import numpy as np
import pytest

from oracle import phipm_oracle as O
import tests.test_oracle_krylov as K
import tests.test_oracle_phi_expm as PE
import tests.test_oracle_phipm as PP


def _aug_transposed(H_m, tau, p):
    return O.__dict__["_orig_aug"](H_m, tau, p).T


def _aug_tau_everywhere(H_m, tau, p):
    m = H_m.shape[0]
    Hh = O.__dict__["_orig_aug"](H_m, 1.0, p)
    return tau * Hh


@pytest.fixture
def orig(monkeypatch):
    monkeypatch.setitem(O.__dict__, "_orig_aug", O.augmented_matrix)
    return monkeypatch


@pytest.mark.parametrize("bad", [_aug_transposed, _aug_tau_everywhere])
def test_augmented_matrix_mistakes(orig, bad):
    orig.setattr(O, "augmented_matrix", bad)
    with pytest.raises(AssertionError):
        PE.test_augmented_matrix_identity(2)


def test_pade_coefficient_mistake(monkeypatch):
    good = O.pade13_coefficients()
    monkeypatch.setattr(O, "pade13_coefficients", lambda: [c * (1.0 + 1e-6 * j) for j, c in enumerate(good)])
    with pytest.raises(AssertionError):
        PE.test_expm_textbook_cases()


def test_squaring_count_mistake(monkeypatch):
    monkeypatch.setattr(O, "squarings", lambda norm1, theta: 0)
    with pytest.raises(AssertionError):
        PE.test_expm_vs_scipy_and_inverse(45.0)


def test_arnoldi_skips_first_projection(monkeypatch):
    def bad(matvec, v, m, bd):
        V = np.zeros((m + 1, v.size))
        H = np.zeros((m + 1, m))
        V[0] = v / np.linalg.norm(v)
        for j in range(m):
            w = matvec(V[j])
            for i in range(1, j + 1):          # i = 0 dropped
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V[j + 1] = w / H[j + 1, j]
        return V, H, m
    monkeypatch.setattr(O, "arnoldi", bad)
    with pytest.raises(AssertionError):
        K.test_arnoldi_relation_and_orthonormality()


def test_lanczos_index_mistake(monkeypatch):
    def bad(matvec, v, m, bd):
        V = np.zeros((m + 1, v.size))
        T = np.zeros((m + 1, m))
        V[0] = v / np.linalg.norm(v)
        for j in range(m):
            w = matvec(V[j])
            T[j, j] = V[j] @ w
            if j > 0:
                w = w - T[j - 1, j - 1] * V[j - 1]   # wrong entry (diagonal instead of t_{j,j-1})
            w = w - T[j, j] * V[j]
            T[j + 1, j] = np.linalg.norm(w)
            if j + 1 < m:
                T[j, j + 1] = T[j + 1, j]
            V[j + 1] = w / T[j + 1, j]
        return V, T, m
    monkeypatch.setattr(O, "lanczos", bad)
    with pytest.raises(AssertionError):
        K.test_lanczos_matches_arnoldi_on_symmetric()


def _attempt_variant(sign=1.0, eps_power=1):
    def attempt(matvec, krylov, v, tau, m, p, bd_abs, theta13=O.DEFAULTS["theta13"]):
        beta = float(np.linalg.norm(v))
        V, H, me = krylov(matvec, v, m, bd_abs)
        E = O.expm_pade13(O.augmented_matrix(H[:me, :me], tau, p), theta13)
        phi_p = E[:me, me + p - 1] if p >= 1 else E[:me, 0]
        phi_p1 = E[:me, me + p]
        h = H[me, me - 1]
        F = tau ** p * beta * (V[:me].T @ phi_p + sign * tau * h * phi_p1[me - 1] * V[me])
        eps = tau ** (p + eps_power) * beta * abs(h) * abs(phi_p1[me - 1])
        return F, eps, me, float(np.max(np.abs(E).sum(axis=0))), beta
    return attempt


def test_corrector_sign_mistake(monkeypatch):
    monkeypatch.setattr(O, "krylov_attempt", _attempt_variant(sign=-1.0))
    with pytest.raises(AssertionError):
        K.test_corrector_and_error_estimate(2, 3e-3, 5)


def test_error_estimate_missing_tau(monkeypatch):
    monkeypatch.setattr(O, "krylov_attempt", _attempt_variant(eps_power=0))
    with pytest.raises(AssertionError):
        K.test_corrector_and_error_estimate(2, 3e-3, 5)


def test_w_recurrence_missing_factorial(monkeypatch):
    def bad(matvec, u, b, t):
        p = len(b) - 1
        W = [u]
        for j in range(1, p + 1):
            wj = matvec(W[j - 1])
            for ell in range(0, p - j + 1):
                wj = wj + (t ** ell) * b[j + ell]          # 1/l! dropped
            W.append(wj)
        return W
    monkeypatch.setattr(O, "w_recurrence", bad)
    with pytest.raises(AssertionError):
        PP.test_diagonal_vs_scalar_phi(4)


def test_step_update_missing_factorial(monkeypatch):
    def bad(F, W, tau):
        return F + sum(tau ** j * W[j] for j in range(len(W) - 1))
    monkeypatch.setattr(O, "step_update", bad)
    with pytest.raises(AssertionError):
        PP.test_laplacian_2d_vs_sine_expansion(32, 3, 1e-8)


def test_omega_without_t_end(monkeypatch):
    monkeypatch.setattr(O, "omega_ratio", lambda eps, tau, t_end, tol: eps / (tau * tol))
    with pytest.raises(AssertionError):
        PP.test_long_horizon_error_budget()


def test_q_hat_printed_inverted(monkeypatch):
    """Eq. (6) as printed (inverted) breaks the hand-computed controller case."""
    orig = O.controller

    def bad(eps, omega, tau, m, mem, prm):
        if mem.rejected and mem.tau_changed and eps > 0 and mem.eps_old > 0:
            q = math.log(tau / mem.tau_old) / math.log(eps / mem.eps_old) - 1.0
            mem.q_hat, mem.q_from_formula = q, True
            mem.rejected, mem.tau_changed = False, False
            _, tn, k, mn = orig(eps, omega, tau, m, mem, prm)
            return q, tn, k, mn
        return orig(eps, omega, tau, m, mem, prm)
    monkeypatch.setattr(O, "controller", bad)
    with pytest.raises(AssertionError):
        PP.test_controller_hand_cases()


def test_phip_that_still_adapts_m(monkeypatch):
    """phip (R20) with the m branch left on is phipm started at m: the fixed-m pin fails."""
    import tests.test_oracle_phip as PH
    monkeypatch.setattr(O, "phip", lambda t_end, A, b, tol=1e-7, symm=-1, m=30, params=None, trace=None:
                        O.phipm(t_end, A, b, tol, symm, dict(params or {}, m_init=m), trace))
    with pytest.raises(AssertionError):
        PH.test_phip_keeps_m_and_meets_tol(6)


def test_w_recurrence_without_the_inhomogeneous_terms(monkeypatch):
    """Eq. (wrecurrence) with the b_{j+l} sums dropped solves u' = Au instead of
    u' = Au + b_1: the Heston pin against the dense augmented exponential fails."""
    import tests.test_oracle_heston as HE

    def bad(matvec, u, b, t):
        W = [u]
        for j in range(1, len(b)):
            W.append(matvec(W[j - 1]))
        return W
    monkeypatch.setattr(O, "w_recurrence", bad)
    with pytest.raises(AssertionError):
        HE.test_heston_small_grid_vs_dense_augmented()
