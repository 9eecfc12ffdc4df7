"""The fixed-dimension variant phip (controller PHIPM_CTRL_FIXED_M) and the Sec. 4.2
nine-point workloads on the CUDA path, against the oracle run with adapt_m off and
against exact truths.  Bar: relative 2-norm error <= 1e-8 (FP64 modes)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import phipm_oracle as O
from oracle import truth as T
from paper_0907_4631_gb300 import phipm as pm
from paper_0907_4631_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-8


def _dev(b):
    return [torch.as_tensor(np.ascontiguousarray(x)).cuda() for x in b]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _solve(s, op, b, t_end, tol, symm):
    u, st, _ = s.solve(t_end, pm.DeviceOperator(op), _dev(b), tol, symm)
    torch.cuda.synchronize()
    return u.cpu().numpy(), st


@pytest.mark.parametrize("prec", ["f64", "f64pair"])
@pytest.mark.parametrize("m", [5, 12])
def test_phip_laplacian_matches_oracle(prec, m):
    """Lanczos path, several steps, rejections at m = 5: the same steps, rejections and
    exponentials as the oracle, every attempt at the fixed m."""
    pr = wl.laplacian_2d_problem(N=16, p=1, t_end=0.05, tol=1e-10, seed=1017)
    s = pm.Phipm(prec, controller=pm.CTRL_FIXED_M, m_init=m)
    s.trace_enable(4096)
    u, st = _solve(s, pr.op, pr.b, pr.t_end, pr.tol, 1)
    tr = s.trace_read()
    ref, rst = O.phip(pr.t_end, pr.op, pr.b, pr.tol, 1, m=m)
    assert _rel(u, ref) <= TOL64
    assert (st["steps"], st["rejects"], st["expms"]) == (rst.steps, rst.rejects, rst.expms)
    assert tr and all(r["m_used"] == m and r["m_req"] == m for r in tr)
    assert np.linalg.norm(u - T.solution_laplacian(2, 16, pr.b, pr.t_end)) <= 2 * pr.tol


@pytest.mark.parametrize("prec,team", [("f64", 1), ("f64pair", 1), ("f64pair", 8), ("f64", 152)])
def test_phip_convdiff_matches_oracle(prec, team):
    """Arnoldi path on one CTA, a cluster and the whole grid (n = 16,900)."""
    pr = wl.convdiff_2d_problem(N=130, p=2, t_end=1e-3, tol=1e-8, seed=2230)
    s = pm.Phipm(prec, controller=pm.CTRL_FIXED_M, m_init=20)
    s.set_team(team)
    u, st = _solve(s, pr.op, pr.b, pr.t_end, pr.tol, 0)
    ref, rst = O.phip(pr.t_end, pr.op, pr.b, pr.tol, 0, m=20)
    assert _rel(u, ref) <= TOL64
    assert st["steps"] == rst.steps and st["rejects"] == rst.rejects


@pytest.mark.parametrize("prec", ["f64", "f64pair"])
@pytest.mark.parametrize("ctrl", [pm.CTRL_PAPER, pm.CTRL_FIXED_M])
def test_nine_point_round_trip(prec, ctrl):
    """e^{-tA} e^{tA} b_0 = b_0 (t = 2, Tol = 1e-14): the forward result matches the oracle,
    and the round trip returns b_0 to the accuracy the reverse amplification allows: the
    reverse pass multiplies the forward pass's rounding error in the top eigenmode by up to
    e^{2 * 12}, about 2e-6 relative per unit roundoff of 2^-53 (IEEE FP64 basis) and 32 times
    that with the 48-bit float-pair basis."""
    A, B, b0, t, tol = wl.nine_point_round_trip()
    s = pm.Phipm(prec, controller=ctrl, m_init=30 if ctrl == pm.CTRL_FIXED_M else 10)
    prm = dict(adapt_m=False, m_init=30) if ctrl == pm.CTRL_FIXED_M else None
    w, _ = _solve(s, A, [b0], t, tol, 1)
    w_ref, _ = O.phipm(t, A, [b0], tol, 1, params=prm)
    assert _rel(w, w_ref) <= TOL64
    r, _ = _solve(s, B, [w], t, tol, 1)
    assert _rel(r, b0) <= (1e-5 if prec == "f64" else 3e-4)


@pytest.mark.parametrize("ctrl", [pm.CTRL_PAPER, pm.CTRL_FIXED_M])
def test_nine_point_phi_sum(ctrl):
    """Experiment 2 stand-in (k <= 4, every b_k = 1, t = 2, Tol = 2^-26)."""
    pr = wl.nine_point_phi_sum_problem()
    s = pm.Phipm("f64pair", controller=ctrl, m_init=30 if ctrl == pm.CTRL_FIXED_M else 10)
    u, st = _solve(s, pr.op, pr.b, pr.t_end, pr.tol, 1)
    fn = O.phip if ctrl == pm.CTRL_FIXED_M else O.phipm
    ref, rst = fn(pr.t_end, pr.op, pr.b, pr.tol, 1)
    assert _rel(u, ref) <= TOL64
    assert st["steps"] == rst.steps and st["rejects"] == rst.rejects


def test_batched_phip():
    """The batched persistent form with the fixed-dimension controller."""
    probs = wl.batched_convdiff_problems(count=6, side_lo=16, side_hi=64, seed0=4990)
    s = pm.Phipm("f64pair", controller=pm.CTRL_FIXED_M, m_init=16)
    ops = [pm.DeviceOperator(p_.op) for p_ in probs]
    us, stats, sts = s.solve_batched([p_.t_end for p_ in probs], ops, [_dev(p_.b) for p_ in probs],
                                     [p_.tol for p_ in probs], [0] * len(probs))
    torch.cuda.synchronize()
    assert all(x == pm.OK for x in sts)
    for p_, u, st in zip(probs, us, stats):
        ref, rst = O.phip(p_.t_end, p_.op, p_.b, p_.tol, 0, m=16)
        assert _rel(u.cpu().numpy(), ref) <= TOL64
        assert st["steps"] == rst.steps
