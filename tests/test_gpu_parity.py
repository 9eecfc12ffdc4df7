"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle and with
exact truths.  Bar: relative 2-norm error <= 1e-8 in FP64 mode and <= 1e-5 in
the FP32 basis mode, the tolerances the method is specified to meet."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import phipm_oracle as O
from oracle import truth as T
from paper_0907_4631_gb300 import phipm as pm
from paper_0907_4631_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-8
TOL32 = 1e-5


_SOLVERS = {}


def _solver(prec):
    if prec not in _SOLVERS:
        _SOLVERS[prec] = pm.Phipm(prec)
    return _SOLVERS[prec]


@pytest.fixture(scope="module", params=["f64", "f64pair"])
def solver64(request):
    """Both FP64-class modes: IEEE FP64 arithmetic, and float pairs on the FP32 pipe."""
    return _solver(request.param)


@pytest.fixture(scope="module")
def solver32():
    return _solver("f32")


def _dev(b):
    return [torch.as_tensor(np.ascontiguousarray(x)).cuda() for x in b]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gpu(solver, pr, symm=None):
    A = pm.DeviceOperator(pr.op)
    u, st, _ = solver.solve(pr.t_end, A, _dev(pr.b), pr.tol, pr.symm if symm is None else symm)
    torch.cuda.synchronize()
    return u.cpu().numpy(), st


@pytest.mark.parametrize("as_csr", [False, True])
def test_c1_laplacian_32(solver64, as_csr):
    """Plain FP64 configuration: 32x32 Laplacian, p=3, t=0.01, tol 1e-8 (Lanczos)."""
    pr = wl.laplacian_2d_problem(as_csr=as_csr)
    u, st = _gpu(solver64, pr, symm=-1)
    ref, rst = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, -1)
    assert _rel(u, ref) <= TOL64
    assert _rel(u, T.solution_laplacian(2, 32, pr.b, pr.t_end)) <= TOL64
    assert st["steps"] == rst.steps and st["rejects"] == rst.rejects


@pytest.mark.parametrize("p", [0, 1, 2, 4])
def test_small_convdiff_cta_path(solver64, p):
    pr = wl.convdiff_2d_problem(N=40, p=p, t_end=1e-3, tol=1e-8, seed=2040 + p)
    u, st = _gpu(solver64, pr)
    ref, rst = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    assert _rel(u, ref) <= TOL64
    assert st["steps"] == rst.steps


@pytest.mark.parametrize("N,p", [(130, 4), (171, 2)])
def test_convdiff_grid_path(solver64, N, p):
    """n = N^2 >= 16384 runs on every SM; N = 171 gives a ragged tail (n not a multiple of 64)."""
    pr = wl.convdiff_2d_problem(N=N, p=p, t_end=1e-3, tol=1e-8, seed=2100 + N)
    u, st = _gpu(solver64, pr)
    ref, rst = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    assert _rel(u, ref) <= TOL64
    assert st["steps"] == rst.steps


def test_laplacian_grid_lanczos(solver64):
    pr = wl.laplacian_2d_problem(N=150, p=2, t_end=2e-3, tol=1e-8, seed=1150)
    u, st = _gpu(solver64, pr, symm=-1)
    assert _rel(u, T.solution_laplacian(2, 150, pr.b, pr.t_end)) <= TOL64


def test_c2_full_size(solver64):
    """FP64 nonsymmetric configuration at full size: 512^2 convection-diffusion, CSR, p=4."""
    pr = wl.convdiff_2d_problem()
    u, st = _gpu(solver64, pr)
    ref, rst = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    assert _rel(u, ref) <= TOL64
    assert st["steps"] >= 1


@pytest.mark.parametrize("N", [24, 40])
def test_f32_laplacian_3d(solver32, N):
    pr = wl.laplacian_3d_problem(N=N, p=2, t_end=1e-4, tol=1e-5, seed=3000 + N)
    u, st = _gpu(solver32, pr)
    ref, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1)
    assert _rel(u, ref) <= TOL32
    assert _rel(u, T.solution_laplacian(3, N, pr.b, pr.t_end)) <= TOL32


def test_c3_full_size_f32(solver32):
    """Precision form at full size: 128^3 Laplacian stencil, FP32 basis, p=2, tol 1e-5,
    checked against the sine eigen-expansion (exact)."""
    pr = wl.laplacian_3d_problem()
    u, st = _gpu(solver32, pr)
    assert _rel(u, T.solution_laplacian(3, 128, pr.b, pr.t_end)) <= TOL32


def test_f32_convdiff_csr(solver32):
    pr = wl.convdiff_2d_problem(N=64, p=3, t_end=1e-3, tol=1e-5, seed=2064)
    u, st = _gpu(solver32, pr)
    ref, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    assert _rel(u, ref) <= TOL32


def test_edge_cases(solver64):
    A = wl.laplacian(2, 6)
    n = A.n
    z = np.zeros(n)
    u, st = _gpu(solver64, wl.Problem("zero", A, [z, z, z], 1e-2, 1e-8, 1))
    assert np.all(u == 0) and st["steps"] == 0
    b1 = wl.normal(4, 1, n)
    u, _ = _gpu(solver64, wl.Problem("b0zero", A, [z, b1], 1e-2, 1e-10, 1))
    ref, _ = O.phipm(1e-2, A, [z, b1], 1e-10, 1)
    assert _rel(u, ref) <= TOL64
    Z = wl.dense_to_csr(np.zeros((5, 5)))
    Z = wl.CSR(5, np.zeros(6, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    bz = [wl.normal(4, k, 5) for k in range(4)]
    u, _ = _gpu(solver64, wl.Problem("Azero", Z, bz, 0.3, 1e-8, -1))
    assert np.allclose(u, sum(0.3 ** k / np.prod(range(1, k + 1)) * bk for k, bk in enumerate(bz)), rtol=1e-14)
    small = wl.random_sparse(3, 5, 3, 1.0)                    # n < m: happy breakdown
    bs = [wl.normal(5, k, 5) for k in range(3)]
    u, _ = _gpu(solver64, wl.Problem("tiny", small, bs, 1.0, 1e-12, -1))
    assert np.allclose(u, T.solution_dense_augmented(wl.csr_to_dense(small), bs, 1.0), rtol=1e-11, atol=1e-12)
    one = wl.dense_to_csr(np.array([[-3.0]]))                  # n = 1
    u, _ = _gpu(solver64, wl.Problem("one", one, [np.array([2.0]), np.array([1.0])], 0.5, 1e-12, -1))
    assert u[0] == pytest.approx(np.exp(-1.5) * 2.0 + 0.5 * T.phi_scalar(1, -1.5) * 1.0, rel=1e-12)


@pytest.mark.parametrize("p", [0, 3])
def test_dense_truth_nonsymmetric(solver64, p):
    A = wl.random_sparse(11, 60, 5, 3.0)
    b = [wl.normal(11, 10 + k, 60) for k in range(p + 1)]
    u, _ = _gpu(solver64, wl.Problem("rs", A, b, 2.0, 1e-10, -1))
    assert np.linalg.norm(u - T.solution_dense_augmented(wl.csr_to_dense(A), b, 2.0)) <= 5e-10


def test_invalid_arguments(solver64):
    pr = wl.laplacian_2d_problem(N=8, p=1)
    A = pm.DeviceOperator(pr.op)
    b = _dev(pr.b)
    for kwargs, bad in [(dict(symm=2), "symm"), (dict(tol=float("nan")), "tol")]:
        _, _, st = solver64.solve(pr.t_end, A, b, check=False, **{"tol": 1e-8, "symm": 1, **kwargs})
        assert st == pm.EINVAL, bad
    _, _, st = solver64.solve(-1.0, A, b, 1e-8, 1, check=False)
    assert st == pm.EINVAL
    _, _, st = solver64.solve(pr.t_end, A, b * 5, 1e-8, 1, check=False)     # p = 9 > 8
    assert st == pm.EINVAL


def test_host_api_matches_device_api(solver64):
    pr = wl.convdiff_2d_problem(N=48, p=2, t_end=1e-3, tol=1e-8, seed=2048)
    u_dev, st_dev = _gpu(solver64, pr)
    u_host, st_host, _ = solver64.solve_host(pr.t_end, pm.HostOperator(pr.op), pr.b, pr.tol, 0)
    st_dev.pop("kernel_ms"), st_host.pop("kernel_ms")
    assert np.array_equal(u_dev, u_host) and st_dev == st_host


def test_deterministic(solver64):
    pr = wl.convdiff_2d_problem(N=140, p=3, t_end=1e-3, tol=1e-8, seed=2140)
    u1, _ = _gpu(solver64, pr)
    u2, _ = _gpu(solver64, pr)
    assert np.array_equal(u1, u2)


def test_batched_small(solver64):
    probs = wl.batched_convdiff_problems(count=6, side_lo=16, side_hi=48, seed0=4900)
    ops = [pm.DeviceOperator(p_.op) for p_ in probs]
    us, stats, sts = solver64.solve_batched([p_.t_end for p_ in probs], ops, [_dev(p_.b) for p_ in probs],
                                            [p_.tol for p_ in probs], [0] * len(probs))
    torch.cuda.synchronize()
    for p_, u, st in zip(probs, us, stats):
        ref, rst = O.phipm(p_.t_end, p_.op, p_.b, p_.tol, 0)
        assert _rel(u.cpu().numpy(), ref) <= TOL64
        assert st["steps"] == rst.steps


def test_pair_mode_agrees_with_native_fp64():
    """The float-pair basis reproduces the IEEE FP64 path on the same inputs: the pair rounding
    (about 2^-48) is amplified only by the cancellation in Eq. (step), far below the 1e-8 bar."""
    pr = wl.convdiff_2d_problem(N=160, p=3, t_end=1e-3, tol=1e-8, seed=2160)
    u64, st64 = _gpu(_solver("f64"), pr)
    u2, st2 = _gpu(_solver("f64pair"), pr)
    assert _rel(u2, u64) <= 1e-9
    assert st64["steps"] == st2["steps"] and st64["krylov_steps"] == st2["krylov_steps"]


@pytest.mark.parametrize("n,prec,team", [(6000, "f64", 1), (6000, "f64", 152), (6000, "f64pair", 8),
                                         (6000, "f32", 4), (6, "f64", 1), (6, "f64pair", 1), (9, "f32", 1),
                                         (4, "f64", 1), (4, "f64pair", 1)])
def test_arnoldi_breakdown_three_eigenvalues(n, prec, team):
    """A diagonal operator with three distinct eigenvalues solved as nonsymmetric
    (Arnoldi): the Krylov space is invariant after three steps, so the fourth candidate
    is rounding noise.  With n = 4 most of that noise lies in the span of the basis: the
    candidate fails the Pythagorean orthogonality check and is projected a second time.  In IEEE
    FP64 the noise falls below the breakdown threshold (R12) and the space stops at
    dimension 3; with float pairs (48-bit basis) or FP32 it can stay above it and the
    solve goes on with directions whose coupling to the problem is at the noise level.
    Teams of 1 to 152 CTAs.  Truth: the scalar phi functions."""
    lams = np.array([-1.0, -5.0, -20.0])[np.arange(n) % 3]
    A = wl.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), lams.copy())
    b = [wl.normal(77, k, n) for k in range(3)]
    s = pm.Phipm(prec)
    s.set_team(team)
    u, st, _ = s.solve(0.7, pm.DeviceOperator(A), _dev(b), 1e-9, 0)
    ref = T.solution_diagonal(lams, b, 0.7)
    assert _rel(u.cpu().numpy(), ref) <= (TOL32 if prec == "f32" else TOL64)
    if prec == "f64":
        assert st["krylov_steps"] <= 4 * max(1, st["expms"])    # the space never grows past dimension 3


@pytest.mark.parametrize("prec,team", [("f64", 1), ("f64", 152), ("f64pair", 1), ("f64pair", 8)])
def test_second_projection_only_when_the_first_loses_most_of_the_vector(prec, team):
    """Selective second Gram-Schmidt pass of the FP64-class bases.  A clustered spectrum
    (eigenvalues in [-1.001, -1]) makes A v nearly parallel to v: the first projection
    removes almost all of each new vector, so every candidate takes its second projection
    (reorth_vectors counts the basis vectors those passes read).  The convection-diffusion
    operator's Krylov vectors keep about 45% of their norm through the first projection,
    so no candidate needs a second one.  Both results match their truths: the scalar phi
    functions, and the oracle's modified Gram-Schmidt Arnoldi."""
    n = 3000
    lams = -(1.0 + 1e-3 * wl.uniform(7001, 0, n))
    A = wl.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), lams.copy())
    b = [wl.normal(7002, k, n) for k in range(3)]
    s = pm.Phipm(prec)
    s.set_team(team)
    u, st, _ = s.solve(2.0, pm.DeviceOperator(A), _dev(b), 1e-10, 0)
    assert _rel(u.cpu().numpy(), T.solution_diagonal(lams, b, 2.0)) <= TOL64
    assert st["reorth_vectors"] > 0 and st["gs_vectors"] > 0
    pr = wl.convdiff_2d_problem(N=48, p=2, t_end=1e-3, tol=1e-8, seed=2048)
    u, st = _gpu(s, pr)
    ref, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    assert _rel(u, ref) <= TOL64
    assert st["reorth_vectors"] == 0 and st["gs_vectors"] > 0


def test_fp32_basis_always_takes_both_passes():
    pr = wl.convdiff_2d_problem(N=48, p=2, t_end=1e-3, tol=1e-5, seed=2049)
    u, st = _gpu(_solver("f32"), pr)
    ref, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    assert _rel(u, ref) <= TOL32
    assert st["reorth_vectors"] > 0


@pytest.mark.parametrize("prec,K", [("f64pair", 2), ("f64pair", 4), ("f64", 8), ("f32", 4)])
def test_batched_cluster_teams(prec, K):
    """Batched form with a thread-block cluster of K CTAs per problem (rows split over the
    cluster, barriers in distributed shared memory): every result matches the oracle,
    including problems too small to give each CTA of the cluster rows."""
    probs = wl.batched_convdiff_problems(count=9, side_lo=6, side_hi=72, seed0=4950)
    if prec == "f32":
        for p_ in probs:
            p_.tol = 1e-5
    s = pm.Phipm(prec)
    s.set_team(K)
    ops = [pm.DeviceOperator(p_.op) for p_ in probs]
    us, stats, sts = s.solve_batched([p_.t_end for p_ in probs], ops, [_dev(p_.b) for p_ in probs],
                                     [p_.tol for p_ in probs], [0] * len(probs))
    torch.cuda.synchronize()
    assert all(x == pm.OK for x in sts)
    for p_, u in zip(probs, us):
        ref, _ = O.phipm(p_.t_end, p_.op, p_.b, p_.tol, 0)
        assert _rel(u.cpu().numpy(), ref) <= (TOL32 if prec == "f32" else TOL64)


def test_batched_graph_replay_sees_new_inputs():
    """The batched launch sequence is captured once and replayed: a second call with the same
    shapes but new right-hand sides, new t_end and new tolerances (descriptors re-read from
    pinned host memory, vectors read from device memory) must give the new answers, and a
    new team size on the same handle (a different launch) must not reuse the graph."""
    s = pm.Phipm("f64pair")
    probs = wl.batched_convdiff_problems(count=5, side_lo=16, side_hi=40, seed0=4970)
    ops = [pm.DeviceOperator(p_.op) for p_ in probs]
    bs = [_dev(p_.b) for p_ in probs]
    batch = s.batch([p_.t_end for p_ in probs], ops, bs, [p_.tol for p_ in probs], [0] * len(probs))
    batch.run()
    first = [u.cpu().numpy().copy() for u in batch.outs]
    for p_, u in zip(probs, first):
        ref, _ = O.phipm(p_.t_end, p_.op, p_.b, p_.tol, 0)
        assert _rel(u, ref) <= TOL64
    # same shapes, new values: b scaled in place on the device, new t_end and tol through a new call
    for b in bs:
        for x in b:
            x.mul_(-0.5)
    t2 = [0.5 * p_.t_end for p_ in probs]
    tol2 = [1e-9] * len(probs)
    us, st, sts = s.solve_batched(t2, ops, bs, tol2, [0] * len(probs), outs=batch.outs)
    torch.cuda.synchronize()
    for p_, u, t, tl in zip(probs, us, t2, tol2):
        ref, _ = O.phipm(t, p_.op, [-0.5 * x for x in p_.b], tl, 0)
        assert _rel(u.cpu().numpy(), ref) <= TOL64
    s.set_team(2)                                      # cluster teams: a new graph
    us, st, sts = s.solve_batched(t2, ops, bs, tol2, [0] * len(probs))
    torch.cuda.synchronize()
    for p_, u, t, tl in zip(probs, us, t2, tol2):
        ref, _ = O.phipm(t, p_.op, [-0.5 * x for x in p_.b], tl, 0)
        assert _rel(u.cpu().numpy(), ref) <= TOL64


@pytest.mark.parametrize("prec,case", [("f64", "lap2d_32"), ("f64pair", "lap2d_150"), ("f32", "lap3d_40"),
                                       ("f64", "lap3d_24")])
def test_stencil_rows_staged_by_tma(prec, case):
    """params.stencil_stage = 1: each stencil product first copies the CTA's rows and the
    grid lines next to them in y into shared memory with one TMA bulk copy (when they fit),
    on one CTA and on the grid; results against the sine expansion."""
    s = pm.Phipm(prec, stencil_stage=1)
    if case == "lap2d_32":
        pr = wl.laplacian_2d_problem()
        ndim, N = 2, 32
    elif case == "lap2d_150":
        pr = wl.laplacian_2d_problem(N=150, p=2, t_end=2e-3, tol=1e-8, seed=1151)
        ndim, N = 2, 150
    elif case == "lap3d_40":
        pr = wl.laplacian_3d_problem(N=40, p=2, t_end=1e-4, tol=1e-5, seed=3040)
        ndim, N = 3, 40
    else:
        pr = wl.laplacian_3d_problem(N=24, p=2, t_end=1e-4, tol=1e-8, seed=3024)
        ndim, N = 3, 24
    u, st = _gpu(s, pr, symm=-1)
    truth = T.solution_laplacian(ndim, N, pr.b, pr.t_end)
    assert _rel(u, truth) <= (TOL32 if prec == "f32" else TOL64)


@pytest.mark.parametrize("team", [1, 4, 152])
def test_pade_exponential_option_matches_the_oracle(team):
    """params.expm_pade = 1: the exponential by the degree-13 Pade approximant, as the paper
    computes it (the default is the degree-18 Taylor form); one CTA, a cluster, the grid."""
    pr = wl.convdiff_2d_problem(N=130, p=3, t_end=1e-3, tol=1e-8, seed=2230)
    ref, rst = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    for pade in (0, 1):
        s = pm.Phipm("f64", expm_pade=pade)
        s.set_team(team)
        u, st = _gpu(s, pr)
        assert _rel(u, ref) <= TOL64
        assert st["steps"] == rst.steps


@pytest.mark.parametrize("prec", ["f64", "f64pair", "f32"])
@pytest.mark.parametrize("team", [1, 152])
def test_output_only_eight_byte_aligned(prec, team):
    """u at an 8-byte (not 16-byte) boundary, on a stencil whose side is a multiple of 4:
    the library reads u as w_0 of the recurrence and writes every accepted step there, so
    it takes the one-row stencil product and the one-row accept step; the result equals
    the aligned solve's up to rounding (the two stencil forms add the neighbours in
    different orders)."""
    tol = TOL32 if prec == "f32" else 1e-8
    pr = wl.laplacian_3d_problem(N=24, p=2, t_end=1e-4, tol=tol, seed=3124)
    s = pm.Phipm(prec)
    s.set_team(team)
    A = pm.DeviceOperator(pr.op)
    b = _dev(pr.b)
    ua, sta, _ = s.solve(pr.t_end, A, b, pr.tol, 1)
    buf = torch.empty(pr.n + 1, dtype=torch.float64, device="cuda")
    uo = buf[1:]
    assert uo.data_ptr() % 16 == 8
    _, sto, _ = s.solve(pr.t_end, A, b, pr.tol, 1, out=uo)
    torch.cuda.synchronize()
    if prec == "f64":
        assert sto["steps"] == sta["steps"]
    assert _rel(uo.cpu().numpy(), ua.cpu().numpy()) <= {"f64": 1e-12, "f64pair": 1e-10, "f32": TOL32}[prec]
    ref, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1)
    assert _rel(uo.cpu().numpy(), ref) <= (TOL32 if prec == "f32" else TOL64)


@pytest.mark.parametrize("action", [0, 1, 2])
@pytest.mark.parametrize("team", [1, 4, 152])
@pytest.mark.parametrize("case", ["lanczos", "arnoldi"])
def test_exponential_action_form_matches_the_oracle(action, team, case):
    """params.expm_action: the phi columns from the action of exp(H_hat) on two unit vectors
    (2), from the full exponential (1), or chosen per attempt by cost (0, the default);
    tridiagonal (Lanczos) and Hessenberg (Arnoldi) H, one CTA, a cluster, the grid.  Each
    meets the oracle (the exponential of the augmented matrix, Eq. hathm) with the same
    steps, and the sine expansion in the symmetric case."""
    if case == "lanczos":
        pr = wl.laplacian_2d_problem()
        ref, rst = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1)
    else:
        pr = wl.convdiff_2d_problem(N=130, p=3, t_end=1e-3, tol=1e-8, seed=2231)
        ref, rst = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0)
    s = pm.Phipm("f64", expm_action=action)
    s.set_team(team)
    u, st = _gpu(s, pr)
    assert _rel(u, ref) <= TOL64
    assert st["steps"] == rst.steps and st["rejects"] == rst.rejects
    if case == "lanczos":
        assert _rel(u, T.solution_laplacian(2, 32, pr.b, pr.t_end)) <= TOL64


@pytest.mark.parametrize("prec", ["f64pair", "f32"])
def test_exponential_action_form_other_precisions(prec):
    tol = TOL32 if prec == "f32" else 1e-8
    pr = wl.laplacian_3d_problem(N=24, p=2, t_end=1e-4, tol=tol, seed=3224)
    ref, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 1)
    for action in (1, 2):
        s = pm.Phipm(prec, expm_action=action)
        u, _ = _gpu(s, pr)
        assert _rel(u, ref) <= (TOL32 if prec == "f32" else TOL64)


@pytest.mark.parametrize("p", [0, 1])
@pytest.mark.parametrize("symm", [1, 0])
def test_exponential_action_form_low_p(p, symm):
    """The action form at p = 0 (H_hat's unit entry only in row 0) and p = 1, for the
    tridiagonal (Lanczos) and Hessenberg (Arnoldi) H, one CTA, against the oracle."""
    if symm:
        A = wl.laplacian(2, 20)
        b = [wl.normal(3300, k, A.n) for k in range(p + 1)]
        t_end, tol = 2e-3, 1e-9
        op = A
    else:
        pr = wl.convdiff_2d_problem(N=40, p=max(p, 1), t_end=1e-3, tol=1e-9, seed=3310)
        op, b, t_end, tol = pr.op, pr.b[: p + 1], pr.t_end, pr.tol
    ref, rst = O.phipm(t_end, op, b, tol, symm)
    s = pm.Phipm("f64", expm_action=2)
    s.set_team(1)
    u, st, _ = s.solve(t_end, pm.DeviceOperator(op), _dev(b), tol, symm)
    torch.cuda.synchronize()
    assert _rel(u.cpu().numpy(), ref) <= TOL64
    assert st["steps"] == rst.steps
