"""Host logic of the learned controller's training data (no GPU): the examples built
from attempt records carry the features the solver computes at the start of a step and
the labels their docstrings define, checked against hand-computed values."""
import math

import numpy as np

from paper_0907_4631_gb300 import learned as L


def _rec(step, attempt, accepted, tau, m, eps, omega, t, rejects_prev=0, m_req=None):
    return dict(problem=0, step=step, attempt=attempt, accepted=accepted, m_req=m if m_req is None else m_req,
                m_used=m, p=2, n=4096, t=t, t_end=1.0, tau=tau, eps=eps, omega=omega, norm_a=100.0, tol=1e-8,
                m_new=float("nan"), source=0, rejects_prev=rejects_prev)


def test_every_step_examples_label_the_supported_tau():
    recs = [
        _rec(0, 0, 0, 0.1, 12, 4e-9, 4.0, 0.0),                  # rejected
        _rec(0, 1, 1, 0.05, 12, 2.5e-10, 0.5, 0.0),              # accepted after a tau change
        _rec(1, 0, 1, 0.06, 12, 3e-10, 0.5, 0.05, rejects_prev=1),
        _rec(2, 0, 1, 0.89, 12, 3e-9, 0.4, 0.11),                # cut to the end of the interval
    ]
    X, T = L.examples_every_step(recs)
    assert X.shape == (2, 8) and T.shape == (2, 2)
    # step 0: q from Eq. (6) on the two attempts at m = 12, clamped to [0, m]
    q0 = min(max(math.log(2.5e-10 / 4e-9) / math.log(0.05 / 0.1) - 1.0, 0.0), 12.0)
    tau0 = 0.05 * (0.8 / 0.5) ** (1.0 / (q0 + 1.0))
    assert np.allclose(T[0], [math.log2(tau0 / 0.1), 12 / 64.0])
    assert np.allclose(X[0], [math.log10(100.0), -8.0, 2.0, math.log10(0.1 * 100.0), 12 / 64.0, 0.0, 0.0,
                              math.log10(4096)])
    # step 1: accepted at once, q = m / 4; omega of step 0's accepted attempt is a feature
    tau1 = 0.06 * (0.8 / 0.5) ** (1.0 / (12 / 4.0 + 1.0))
    assert np.allclose(T[1], [math.log2(tau1 / 0.06), 12 / 64.0])
    assert np.isclose(X[1][5], math.log10(0.5)) and X[1][6] == 1.0


def test_every_step_examples_skip_zero_estimates():
    recs = [_rec(0, 0, 1, 0.1, 5, 0.0, 0.0, 0.0), _rec(1, 0, 1, 0.2, 5, 1e-10, 0.3, 0.1)]
    X, T = L.examples_every_step(recs)
    assert X.shape[0] == 1 and np.isclose(X[0][5], -6.0)     # omega 0 floored at 1e-6
