"""Matrix-free operators on the GPU (Sec. 3.5: A given as a function computing A x),
through the C ABI's PHIPM_OP_FUNCTION kind, against the oracle's Operator kind
"function" (oracle/matrix_free.py) and the sine expansion."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import phipm_oracle as O
from oracle import truth as T
from oracle.matrix_free import VarCoefConvDiffOperator
from paper_0907_4631_gb300 import phipm as pm
from paper_0907_4631_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-8
TOL32 = 1e-5


def _dev(b):
    return [torch.as_tensor(np.ascontiguousarray(x)).cuda() for x in b]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,team", [("f64", 1), ("f64", 152), ("f64pair", 1), ("f64pair", 4), ("f32", 1)])
@pytest.mark.parametrize("ndim,N", [(2, 48), (3, 14)])
def test_variable_coefficient_operator_matches_the_oracle(prec, team, ndim, N):
    """Variable diffusivity and a rotating velocity field (nonsymmetric, Arnoldi); the
    norm bound computed on the device; teams of one CTA, a cluster and the grid."""
    tol = TOL32 if prec == "f32" else 1e-8
    pr = wl.varcoef_convdiff_problem(ndim=ndim, N=N, speed=20.0, p=2, t_end=5e-3, tol=tol, seed=6100 + N)
    s = pm.Phipm(prec)
    s.set_team(team)
    u, st, _ = s.solve(pr.t_end, pm.DeviceOperator(pr.op), _dev(pr.b), pr.tol, 0)
    ref, rst = O.phipm(pr.t_end, VarCoefConvDiffOperator(pr.op), pr.b, pr.tol, 0)
    assert _rel(u.cpu().numpy(), ref) <= (TOL32 if prec == "f32" else TOL64)
    if prec == "f64":
        assert st["steps"] == rst.steps


def test_caller_bound_and_symmetric_declaration():
    """A caller-supplied ||A||_inf bound (the oracle's exact value) gives the device-computed
    solve's result; without convection, symm = 1 runs Lanczos and meets the sine expansion
    for constant kappa (A = c Laplacian at time c t)."""
    pr = wl.varcoef_convdiff_problem(ndim=2, N=40, speed=20.0, p=2, t_end=1e-3, tol=1e-8, seed=6200)
    s = pm.Phipm("f64")
    u0, st0, _ = s.solve(pr.t_end, pm.DeviceOperator(pr.op), _dev(pr.b), pr.tol, 0)
    pr.op.norm_bound = VarCoefConvDiffOperator(pr.op).norm_inf
    u1, st1, _ = s.solve(pr.t_end, pm.DeviceOperator(pr.op), _dev(pr.b), pr.tol, 0)
    assert _rel(u1.cpu().numpy(), u0.cpu().numpy()) <= 1e-12 and st1["steps"] == st0["steps"]
    N, c = 40, 1.7
    data = wl.varcoef_convdiff(2, N, 0.0, seed=6201)
    data.kappa = np.full(N * N, c)
    b = [wl.normal(6202, k, N * N) for k in range(3)]
    u, st, _ = s.solve(0.01, pm.DeviceOperator(data), _dev(b), 1e-9, 1)
    ut = T.solution_laplacian(2, N, [bk / c ** k for k, bk in enumerate(b)], c * 0.01)
    assert _rel(u.cpu().numpy(), ut) <= TOL64
    assert st["gs_vectors"] == 0                          # Lanczos: no Gram-Schmidt passes


def test_function_operator_in_a_batch():
    """Batched form with matrix-free problems of different grids next to a CSR problem."""
    probs = [wl.varcoef_convdiff_problem(ndim=2, N=N, speed=10.0 * k, p=1 + k, t_end=1e-3, tol=1e-8, seed=6300 + k)
             for k, N in enumerate((24, 40, 33))]
    probs.append(wl.convdiff_2d_problem(N=30, p=2, t_end=1e-3, tol=1e-8, seed=6310))
    s = pm.Phipm("f64pair")
    us, stats, sts = s.solve_batched([p_.t_end for p_ in probs], [pm.DeviceOperator(p_.op) for p_ in probs],
                                     [_dev(p_.b) for p_ in probs], [p_.tol for p_ in probs], [0] * len(probs))
    torch.cuda.synchronize()
    assert all(x == pm.OK for x in sts)
    for p_, u in zip(probs, us):
        op = VarCoefConvDiffOperator(p_.op) if hasattr(p_.op, "fields") else p_.op
        ref, _ = O.phipm(p_.t_end, op, p_.b, p_.tol, 0)
        assert _rel(u.cpu().numpy(), ref) <= TOL64


def test_function_operator_rejects_bad_descriptors():
    pr = wl.varcoef_convdiff_problem(ndim=2, N=16, seed=6400)
    A = pm.DeviceOperator(pr.op)
    s = pm.Phipm("f64")
    A.c.fn.field[0] = 0                                   # no diffusivity field
    _, _, st = s.solve(pr.t_end, A, _dev(pr.b), pr.tol, 0, check=False)
    assert st == pm.EINVAL
    A = pm.DeviceOperator(pr.op)
    A.c.fn.fn = 7                                         # unknown function
    _, _, st = s.solve(pr.t_end, A, _dev(pr.b), pr.tol, 0, check=False)
    assert st == pm.EINVAL
