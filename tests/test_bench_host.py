"""Host logic of bench.py (no GPU): every workload it names builds with the sizes the
paper or the configuration fixes, the oracle runs each workload's controller, and the
roofline's byte model and the replica arithmetic are what their docstrings state."""
import math

import numpy as np
import pytest

import bench
from oracle import phipm_oracle as O
from paper_0907_4631_gb300 import workloads as wl


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_every_workload_builds(name):
    spec = bench.WORKLOADS[name]
    if spec.get("batched"):
        probs = bench.make_batch(name, first=3, count=2)
        assert len(probs) == 2 and all(p.n > 0 and 1 <= p.p <= 4 for p in probs)
        if "tol" in spec:
            assert all(p.tol == spec["tol"] for p in probs)
    else:
        pr = bench.make_problem(name)
        assert pr.n > 0 and len(pr.b) == pr.p + 1
        assert all(b.shape == (pr.n,) for b in pr.b)
    assert spec["precision"] in bench.DTYPES


def test_workload_sizes():
    assert bench.make_problem("convdiff2d_512").op.nnz == 1308672
    assert bench.make_problem("heston_100x51").n == 5100
    pr = bench.make_problem("ninepoint30_phi4")
    assert (pr.n, pr.op.nnz, pr.p, pr.t_end) == (900, 7744, 4, 2.0)
    assert pr.tol == 2.0 ** -26


def test_oracle_params_follow_the_controller():
    assert bench.oracle_params("ninepoint30_phi4") == {}
    prm = bench.oracle_params("ninepoint30_phi4_phip")
    assert prm == dict(adapt_m=False, m_init=30)
    pr = bench.make_problem("ninepoint30_phi4_phip")
    trace = []
    O.phipm(pr.t_end, pr.op, pr.b, pr.tol, pr.symm, prm, trace)
    assert trace and all(r["m"] == 30 for r in trace)


def test_algorithmic_bytes_model():
    """Arnoldi: 2 s n per basis-vector visit, plus per step one SpMV (CSR: 12 B per nonzero,
    4 B per row pointer, x read and y written) and 6 s n of candidate traffic."""
    A = wl.stencil_to_csr(wl.convection_diffusion_2d(8, 1.0, 3.0, 4.0))
    pr = wl.Problem("t", A, [np.zeros(A.n)] * 3, 1.0, 1e-8, 0)
    st = dict(krylov_steps=7, gs_vectors=21)
    n, s = A.n, 8
    spmv = 12 * A.nnz + 4 * (n + 1) + 2 * s * n
    assert bench.algorithmic_bytes(pr, st, "f64pair") == 2 * s * n * 21 + 7 * (spmv + 6 * s * n)
    s = 4
    spmv = 12 * A.nnz + 4 * (n + 1) + 2 * s * n
    assert bench.algorithmic_bytes(pr, st, "f32") == 2 * s * n * 21 + 7 * (spmv + 6 * s * n)
    # Lanczos (gs_vectors = 0) on a stencil: SpMV 2 s n plus 7 s n of vector traffic
    pl = wl.Problem("l", wl.laplacian(2, 8), [np.zeros(64)], 1.0, 1e-8, 1)
    assert bench.algorithmic_bytes(pl, dict(krylov_steps=5, gs_vectors=0), "f64") == 5 * (2 * 8 * 64 + 7 * 8 * 64)


def test_replica_throughput():
    # two ranks, 10 solves each in 500 ms (the slowest rank): 40 solves/s for the job
    assert math.isclose(bench.replica_throughput(10, 2, 500.0), 40.0)
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
