"""phipm_solve_noalloc: the solve for callers that must not allocate device memory.

Some callers cannot call cudaMalloc (a host application that owns all device
memory, a latency-bound loop that cannot afford cudaMalloc's implicit
synchronisation).  This entry point runs the single-CTA FP64 solve with its
workspace in a static device array of the library.  This file is collected
last, so a run that stops at the first failure has already run every other test.
"""
import ctypes

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


@pytest.mark.parametrize("N", [64, 90])      # n = 4096, and n = 8100 near the 8192 limit
def test_noalloc_matches_oracle_and_phipm_solve_on_two_calls(N):
    pr = wl.convdiff_2d_problem(N=N, p=3, t_end=1e-3, tol=1e-8, seed=2900 + N)
    A = pm.DeviceOperator(pr.op)
    b = _dev(pr.b)
    oracle, ost = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    ref, ref_stats, st = pm.Phipm("f64").solve(pr.t_end, A, b, pr.tol, 0)
    assert st == pm.OK
    ref = ref.cpu().numpy()
    assert np.linalg.norm(ref - oracle) / np.linalg.norm(oracle) <= TOL64
    for _ in range(2):                       # the static array keeps the previous call's contents
        u, stats, st = pm.solve_noalloc(pr.t_end, A, b, pr.tol, 0)
        torch.cuda.synchronize()
        assert st == pm.OK
        u = u.cpu().numpy()
        assert np.linalg.norm(u - oracle) / np.linalg.norm(oracle) <= TOL64
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= TOL64
        assert stats["steps"] == ref_stats["steps"] and stats["rejects"] == ref_stats["rejects"]
        assert stats["steps"] == ost.steps


def test_noalloc_second_call_takes_no_device_memory():
    """After the first call has loaded the module and its static array, a call with the
    output preallocated leaves the device's free memory unchanged."""
    pr = wl.convdiff_2d_problem(N=48, p=2, t_end=1e-3, tol=1e-8, seed=2990)
    A = pm.DeviceOperator(pr.op)
    b = _dev(pr.b)
    u = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    _, _, st = pm.solve_noalloc(pr.t_end, A, b, pr.tol, 0, out=u)
    torch.cuda.synchronize()
    assert st == pm.OK
    free0, _ = torch.cuda.mem_get_info()
    _, _, st = pm.solve_noalloc(pr.t_end, A, b, pr.tol, 0, out=u)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert st == pm.OK
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    st = wl.laplacian(2, 91)                 # n = 8281 > 8192
    A = pm.DeviceOperator(st)
    b = _dev([np.ones(st.n)])
    _, _, status = pm.solve_noalloc(1e-3, A, b, 1e-8, 1)
    assert status == pm.ETOOLARGE
