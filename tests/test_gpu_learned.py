"""The learned controller's kernels against the FP64 CPU oracle of the network,
attempt traces against the solver's statistics, and the trained controller on a
held-out set against the paper's controller."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_oracle as M
from oracle import phipm_oracle as O
from paper_0907_4631_gb300 import learned as L
from paper_0907_4631_gb300 import phipm as pm
from paper_0907_4631_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    return pm.Phipm("f64pair")


def _rand_problem(n_rows, seed):
    w = M.init_weights(seed)
    w[M.OFF_B1:M.OFF_W2] = wl.normal(seed, 7, 64) * 0.1
    w[M.OFF_B2:M.OFF_W3] = wl.normal(seed, 8, 64) * 0.1
    X = wl.normal(seed, 1, n_rows * 8).reshape(n_rows, 8)
    T = wl.normal(seed, 2, n_rows * 2).reshape(n_rows, 2)
    return w, X, T


@pytest.mark.parametrize("n_rows", [1, 37, 1000])
def test_mlp_forward_and_gradient_match_oracle(solver, n_rows):
    w, X, T = _rand_problem(n_rows, 40 + n_rows)
    wt = torch.as_tensor(w.astype(np.float32)).cuda()
    Xt = torch.as_tensor(X.astype(np.float32)).cuda()
    Tt = torch.as_tensor(T.astype(np.float32)).cuda()
    # the oracle sees exactly the FP32 values the kernels see
    w32, X32, T32 = (a.astype(np.float32).astype(np.float64) for a in (w, X, T))
    y_ref, _ = M.forward(w32, X32)
    y = solver.mlp_forward(wt, Xt).cpu().numpy()
    assert np.linalg.norm(y - y_ref) <= 1e-5 * np.linalg.norm(y_ref)
    loss_ref, g_ref = M.loss_and_grad(w32, X32, T32)
    g, loss = solver.mlp_grad(wt, Xt, Tt)
    g = g.cpu().numpy()
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    for lo, hi in [(M.OFF_W1, M.OFF_B1), (M.OFF_W2, M.OFF_B2), (M.OFF_W3, M.OFF_B3), (M.OFF_B3, M.N_PARAMS)]:
        assert np.linalg.norm(g[lo:hi] - g_ref[lo:hi]) <= 1e-4 * np.linalg.norm(g_ref[lo:hi]) + 1e-9


def test_mlp_adam_matches_oracle(solver):
    w, X, T = _rand_problem(256, 77)
    wt = torch.as_tensor(w.astype(np.float32)).cuda()
    m = torch.zeros_like(wt)
    v = torch.zeros_like(wt)
    Xt = torch.as_tensor(X.astype(np.float32)).cuda()
    Tt = torch.as_tensor(T.astype(np.float32)).cuda()
    losses = solver.mlp_train(wt, m, v, Xt, Tt, 5, 0, 1e-3)
    wr, mr, vr = w.astype(np.float32).astype(np.float64), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    X32, T32 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    ref_losses = []
    for t in range(1, 6):
        l, g = M.loss_and_grad(wr, X32, T32)
        ref_losses.append(l)
        wr, mr, vr = M.adam_step(wr, g, mr, vr, t, lr=1e-3)
    assert np.allclose(losses, ref_losses, rtol=1e-4)
    assert np.linalg.norm(wt.cpu().numpy() - wr) <= 1e-4 * np.linalg.norm(wr)


def test_traces_agree_with_stats(solver):
    pr = wl.convdiff_2d_problem(N=40, p=3, t_end=1e-3, tol=1e-8, seed=2240)
    solver.set_controller(0)
    solver.trace_enable(4096)
    A = pm.DeviceOperator(pr.op)
    u, st, _ = solver.solve(pr.t_end, A, [torch.as_tensor(x).cuda() for x in pr.b], pr.tol, 0)
    recs = solver.trace_read()
    solver.trace_enable(0)
    assert len(recs) == st["expms"]
    assert sum(r["accepted"] for r in recs) == st["steps"]
    acc = [r for r in recs if r["accepted"]]
    assert sum(r["tau"] for r in acc) == pytest.approx(pr.t_end, rel=1e-13)
    for r in acc:                        # omega <= delta on every accepted attempt
        assert r["omega"] <= 1.2 and r["eps"] <= 1.2 * r["tau"] * pr.tol / pr.t_end * (1 + 1e-12)
    trace = []
    O.phipm(pr.t_end, pr.op, pr.b, pr.tol, 0, trace=trace)
    assert [round(r["tau"], 15) for r in recs] == [round(r["tau"], 15) for r in trace]
    assert [r["m_used"] for r in recs] == [r["m"] for r in trace]


def test_learned_controller_on_held_out_problems(solver):
    """Train on traces of configuration-1..3 variants, then solve held-out Peclet problems
    with the paper's controller, the learned first-step proposal and the learned
    every-step proposal (eight results of each checked against the oracle):
    the error estimate still judges every attempt, so accuracy stays at tolerance; the
    learned first proposal cuts the rejected attempts (877 -> 152 in the last measured run),
    the attempts overall (1390 -> 732) and the batch's solve time.  The trajectories, and so
    the training set, move with rounding-level changes of the kernels, so the bounds keep
    a margin below the measured effect."""
    probs = L.training_problems(count=768, seed0=7000)
    recs = L.collect_traces(solver, probs)
    X, T = L.examples_from_traces(recs)
    assert X.shape[0] > 400
    blob, losses = L.train(solver, X, T, iters=1500, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]
    # a separate handle with a step budget: a failure shows as PHIPM_EMAXSTEPS, not a long run
    solver = pm.Phipm("f64pair", max_steps=5000, max_rejects=5000)
    held = wl.peclet_convdiff_problems(count=152, N=128, seed0=5900)
    ops = [pm.DeviceOperator(p_.op) for p_ in held]
    bs = [[torch.as_tensor(x).cuda() for x in p_.b] for p_ in held]
    batch = solver.batch([p_.t_end for p_ in held], ops, bs, [p_.tol for p_ in held], [0] * len(held))

    def run(controller):
        solver.set_controller(controller)
        ms = []
        for _ in range(3):
            batch.run()
            ms.append(batch.stats()[0]["kernel_ms"])
        return [u.cpu().numpy() for u in batch.outs], batch.stats(), min(ms)
    u0, st0, ms0 = run(0)
    solver.set_controller_weights(blob)
    u1, st1, ms1 = run(1)
    # the controller that proposes every step (a network trained on per-step labels);
    # measured to cut rejects but take smaller steps, so it is checked for accuracy here
    # and its counters are reported, not asserted to win
    X3, T3 = L.examples_every_step(recs)
    blob3, losses3 = L.train(solver, X3, T3, iters=1500, lr=3e-3)
    assert losses3[-1] < 0.5 * losses3[0]
    solver.set_controller_weights(blob3)
    u3, st3, ms3 = run(3)
    solver.set_controller(0)
    for k in range(0, 152, 19):                  # eight held-out problems against the oracle
        ref, _ = O.phipm(held[k].t_end, held[k].op, held[k].b, held[k].tol, 0)
        for u in (u0[k], u1[k], u3[k]):
            assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= 1e-8
    print(f"every-step proposals: attempts {sum(s['expms'] for s in st3)}, rejects "
          f"{sum(s['rejects'] for s in st3)}, steps {sum(s['steps'] for s in st3)}, Gram-Schmidt vectors "
          f"{sum(s['gs_vectors'] for s in st3)}, batch ms {ms3:.2f}")
    att0 = sum(s["expms"] for s in st0)
    att1 = sum(s["expms"] for s in st1)
    print(f"held-out attempts: plain {att0}, learned {att1}; rejects {sum(s['rejects'] for s in st0)} -> "
          f"{sum(s['rejects'] for s in st1)}; steps {sum(s['steps'] for s in st0)} -> "
          f"{sum(s['steps'] for s in st1)}; Gram-Schmidt vectors {sum(s['gs_vectors'] for s in st0)} -> "
          f"{sum(s['gs_vectors'] for s in st1)}; batch ms {ms0:.2f} -> {ms1:.2f}")
    rej0 = sum(s["rejects"] for s in st0)
    rej1 = sum(s["rejects"] for s in st1)
    assert rej1 < 0.5 * rej0
    assert att1 < 0.6 * att0
    assert ms1 < ms0
