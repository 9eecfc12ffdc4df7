"""The bounded device-side waits give up with PHIPM_ETIMEOUT instead of hanging.

Every team barrier (cooperative grid, thread-block cluster) spins on an arrival
counter for at most params.timeout_cycles clock cycles.  With a limit of one
cycle, the first CTA that has to wait at all gives up, sets the launch's error
word, and every CTA leaves through the status path within 16 further polls (the
error word is checked every 16 polls; no wait is unbounded).  Nothing here faults
or hangs the GPU: the waits end by themselves, the kernel returns, and the same
handle then solves normally with the default limit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import phipm_oracle as O
from paper_0907_4631_gb300 import phipm as pm
from paper_0907_4631_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-8


def _dev(b):
    return [torch.as_tensor(np.ascontiguousarray(x)).cuda() for x in b]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _set_timeout(solver, cycles):
    solver.params.timeout_cycles = int(cycles)
    solver._check(pm.lib().phipm_set_params(solver.h, pm.ctypes.byref(solver.params)))


def test_grid_barrier_timeout_then_normal_solve():
    """A 16-CTA cooperative grid solve with a one-cycle wait limit returns ETIMEOUT; the
    same handle then solves the problem with the default limit and matches the oracle."""
    pr = wl.convdiff_2d_problem(N=96, p=2, t_end=1e-3, tol=1e-8, seed=6096)
    s = pm.Phipm("f64pair")
    s.set_team(16)                    # more than 8 CTAs: a cooperative grid, not a cluster
    default = int(s.params.timeout_cycles)
    A = pm.DeviceOperator(pr.op)
    b = _dev(pr.b)
    _set_timeout(s, 1)
    _, _, st = s.solve(pr.t_end, A, b, pr.tol, 0, check=False)
    torch.cuda.synchronize()
    assert st == pm.ETIMEOUT, s.last_error()
    _set_timeout(s, default)
    u, stats, st = s.solve(pr.t_end, A, b, pr.tol, 0)
    torch.cuda.synchronize()
    assert st == pm.OK
    ref, rst = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    assert _rel(u.cpu().numpy(), ref) <= TOL64
    assert stats["steps"] == rst.steps


def test_cluster_batch_timeout_statuses_then_normal_batch():
    """A batch on clusters of 4 CTAs with a one-cycle wait limit: the call returns
    ETIMEOUT, no problem that a team never took reports OK (they report ENOTRUN), every
    problem reported OK matches the oracle, and the next call with the default limit
    (a newly captured launch) solves every problem."""
    probs = wl.batched_convdiff_problems(count=12, side_lo=24, side_hi=64, seed0=6200)
    s = pm.Phipm("f64pair")
    s.set_team(4)
    default = int(s.params.timeout_cycles)
    ops = [pm.DeviceOperator(p_.op) for p_ in probs]
    bs = [_dev(p_.b) for p_ in probs]
    args = ([p_.t_end for p_ in probs], ops, bs, [p_.tol for p_ in probs], [0] * len(probs))
    _set_timeout(s, 1)
    us, _, sts = s.solve_batched(*args, check=False)
    torch.cuda.synchronize()
    assert any(x != pm.OK for x in sts)
    assert all(x in (pm.OK, pm.ETIMEOUT, pm.ENOTRUN) for x in sts), sts
    for p_, u, x in zip(probs, us, sts):
        if x == pm.OK:
            ref, _ = O.phipm(p_.t_end, p_.op, p_.b, p_.tol, 0)
            assert _rel(u.cpu().numpy(), ref) <= TOL64
    _set_timeout(s, default)
    us, _, sts = s.solve_batched(*args)
    torch.cuda.synchronize()
    assert all(x == pm.OK for x in sts)
    for p_, u in zip(probs, us):
        ref, _ = O.phipm(p_.t_end, p_.op, p_.b, p_.tol, 0)
        assert _rel(u.cpu().numpy(), ref) <= TOL64
