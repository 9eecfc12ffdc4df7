"""The learned (tau, m) controller: data from attempt traces, training on the GPU.

Flow (every numerical step of training and solving runs in libphipm's kernels;
this module builds arrays and calls the library):
  1. solve a family of training problems with the paper's controller and
     attempt traces enabled (phipm_trace_enable);
  2. turn each solve into one example: the features the solver computes at
     the start of the first step (where Algorithm 3 starts from the heuristic
     tau of Eq. (tau_0) and m_init) and a hindsight label (tau*, m*), given as
     log2(tau* / tau_0) and m* / 64:
       - first step with rejected attempts: the accepted tau, and the m of
         Eq. (3) evaluated on the accepted attempt's error (the smallest m the
         error model expects to meet the tolerance at that tau, at most
         halving the accepted m, which the controller reached by growing m
         in steps of 4/3 and usually overshot);
       - first step accepted at once: the (tau, m) the paper's controller
         proposes right after it (its estimate from a measured error), unless
         that proposal was cut to the end of the interval;
     For the controller that proposes every step (examples_every_step) each
     step gives an example, labelled with the largest tau its own accepted
     attempt supports (Eq. 2 with the margin gamma);
  3. standardise, train the 8-64-64-2 GELU network with phipm_mlp_train
     (full-batch Adam, mean squared error);
  4. install the blob (weights + standardisation) with
     phipm_set_controller_weights and solve with params.controller = 1 (first
     step) or 3 (every step).

The feature definition must match the solver's (csrc/phipm_engine.cuh, learned
proposal block):
  log10(||A||_inf t_end), log10(Tol), p, log10(tau_start ||A||_inf), m_start / 64,
  log10(omega of the previous accepted attempt, floored at 1e-6; 1 before the
  first step), rejected attempts in the previous step, log10(n).
At the first step the last three but one are constants (m_init / 64, 0, 0).
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as wl

N_FEATURES = 8


# --------------------------------------------------------------------------------------
# training problems: seeded variants of the three single-problem configurations
# --------------------------------------------------------------------------------------
def training_problems(count: int = 768, seed0: int = 7000) -> list:
    """Variants of the 2D Laplacian (config 1), the convection-diffusion family of
    config 2 (velocities spanning Peclet numbers 1..1e3) and the 3D Laplacian of
    config 3.  Grid sides are drawn log-uniformly up to 160 (2D Laplacian), 256
    (convection-diffusion) and 40 (3D), so that n spans 256..65536."""
    probs = []
    for i in range(count):
        s = seed0 + i
        kind = i % 3
        u = wl.uniform(s, 1, 6)
        if kind == 0:
            N = int(16 * 10 ** u[0])
            p = int(u[1] * 5) % 5
            t_end = 0.01 * 10 ** (2 * u[2] - 1)
            tol = 10 ** (-10 + 5 * u[3])
            st = wl.laplacian(2, N)
            b = [wl.normal(s, 100 + k, st.n) for k in range(p + 1)]
            probs.append(wl.Problem(f"tr_lap2_{i}", wl.stencil_to_csr(st), b, t_end, tol, 1, meta=dict(seed=s)))
        elif kind == 1:
            N = int(16 * 16 ** u[0])
            p = 1 + int(u[1] * 4) % 4
            t_end = 1e-3 * 10 ** (2 * u[2] - 1)
            tol = 10 ** (-10 + 4 * u[3])
            speed = 10 ** (3 * u[4])
            ang = 2 * math.pi * u[5]
            st = wl.convection_diffusion_2d(N, 1.0, speed * math.cos(ang), speed * math.sin(ang))
            b = [wl.normal(s, 100 + k, st.n) for k in range(p + 1)]
            probs.append(wl.Problem(f"tr_cd_{i}", wl.stencil_to_csr(st), b, t_end, tol, 0, meta=dict(seed=s)))
        else:
            N = int(8 * 5 ** u[0])
            p = int(u[1] * 4) % 4
            t_end = 1e-4 * 10 ** (2 * u[2] - 1)
            tol = 10 ** (-9 + 4 * u[3])
            st = wl.laplacian(3, N)
            b = [wl.uniform(s, 100 + k, st.n, -1.0, 1.0) for k in range(p + 1)]
            probs.append(wl.Problem(f"tr_lap3_{i}", wl.stencil_to_csr(st), b, t_end, tol, 1, meta=dict(seed=s)))
    return probs


# --------------------------------------------------------------------------------------
# traces -> examples
# --------------------------------------------------------------------------------------
def examples_from_traces(records: list) -> tuple:
    """(X_raw [k x 8], T_raw [k x 2]) from attempt records of one or more solves:
    one example per solve, from its first step (the step the learned proposal
    replaces)."""
    by_prob: dict = {}
    for r in records:
        if r["step"] <= 1:
            by_prob.setdefault(r["problem"], []).append(r)
    X, T = [], []
    for prob, recs in by_prob.items():
        first = sorted((r for r in recs if r["step"] == 0), key=lambda r: r["attempt"])
        nxt = sorted((r for r in recs if r["step"] == 1), key=lambda r: r["attempt"])
        acc = [r for r in first if r["accepted"]]
        if not first or not acc or first[0]["attempt"] != 0:
            continue
        r0, ra = first[0], acc[-1]
        if len(first) > 1:
            # accepted tau; m_new of Eq. (3) from the accepted attempt (at most halving m)
            mn = ra["m_new"]
            m_lab = ra["m_used"] if not math.isfinite(mn) else min(ra["m_used"], max(math.ceil(mn),
                                                                                      ra["m_used"] // 2, 1))
            label = (ra["tau"], m_lab)
        elif nxt and nxt[0]["attempt"] == 0 and nxt[0]["t"] + nxt[0]["tau"] < nxt[0]["t_end"] * (1.0 - 1e-12):
            label = (nxt[0]["tau"], nxt[0]["m_req"])
        else:
            continue
        na = r0["norm_a"]
        if not (na > 0 and r0["tau"] > 0 and label[0] > 0):
            continue
        x = [math.log10(na * r0["t_end"]), math.log10(r0["tol"]), float(r0["p"]), math.log10(r0["tau"] * na),
             r0["m_req"] / 64.0, 0.0, float(r0["rejects_prev"]), math.log10(r0["n"])]
        t = [math.log2(label[0] / r0["tau"]), label[1] / 64.0]
        if all(math.isfinite(v) for v in x + t):
            X.append(x)
            T.append(t)
    return np.asarray(X, dtype=np.float64).reshape(-1, N_FEATURES), np.asarray(T, dtype=np.float64).reshape(-1, 2)


def _q_estimate(attempts: list) -> float:
    """q of Eq. (6) from two attempts of a step at the same m and different tau (the
    error model eps ~ tau^(q+1)), else m / 4 as Algorithm 4 starts; clamped to [0, m]."""
    acc = attempts[-1]
    m = acc["m_used"]
    for r in reversed(attempts[:-1]):
        if r["m_used"] == m and r["tau"] != acc["tau"] and r["eps"] > 0 and acc["eps"] > 0:
            q = math.log(acc["eps"] / r["eps"]) / math.log(acc["tau"] / r["tau"]) - 1.0
            if math.isfinite(q):
                return min(max(q, 0.0), float(m))
    return m / 4.0


def examples_every_step(records: list, gamma: float = 0.8) -> tuple:
    """(X_raw, T_raw) for the controller that proposes the first attempt of every step
    (PHIPM_CTRL_LEARNED_STEPS): one example per step, features at the step's start
    (the tau and m Algorithm 4 carried into it, omega of the previous accepted attempt,
    the previous step's rejects) and as label the largest tau the step's own accepted
    attempt supports with the margin gamma of Eq. (2), tau* = tau_acc (gamma /
    omega_acc)^(1/(q+1)) with q from the step's attempts (Eq. 6) or m / 4, together
    with the accepted m.  Unlike the accepted tau, tau* is not biased below what the
    step could take, so the proposals do not shrink from step to step.  Steps cut to
    the end of the interval and steps with a zero estimate give no example."""
    by_prob: dict = {}
    for r in records:
        by_prob.setdefault(r["problem"], {}).setdefault(r["step"], []).append(r)
    X, T = [], []
    for prob, steps in by_prob.items():
        omega_prev = 1.0
        for k in sorted(steps):
            att = sorted(steps[k], key=lambda r: r["attempt"])
            acc = [r for r in att if r["accepted"]]
            if not acc or att[0]["attempt"] != 0:
                break
            r0, ra = att[0], acc[-1]
            upto = att[:att.index(ra) + 1]
            last = ra["t"] + ra["tau"] >= ra["t_end"] * (1.0 - 1e-12)
            na = r0["norm_a"]
            if not last and ra["omega"] > 0 and na > 0 and r0["tau"] > 0:
                q = _q_estimate(upto)
                tau_star = ra["tau"] * (gamma / ra["omega"]) ** (1.0 / (q + 1.0))
                x = [math.log10(na * r0["t_end"]), math.log10(r0["tol"]), float(r0["p"]),
                     math.log10(r0["tau"] * na), r0["m_req"] / 64.0, math.log10(max(omega_prev, 1e-6)),
                     float(r0["rejects_prev"]), math.log10(r0["n"])]
                t = [math.log2(tau_star / r0["tau"]), ra["m_used"] / 64.0]
                if all(math.isfinite(v) for v in x + t):
                    X.append(x)
                    T.append(t)
            omega_prev = ra["omega"]
    return np.asarray(X, dtype=np.float64).reshape(-1, N_FEATURES), np.asarray(T, dtype=np.float64).reshape(-1, 2)


def standardise(X: np.ndarray, T: np.ndarray):
    xm, xs = X.mean(axis=0), X.std(axis=0)
    xs = np.where(xs < 1e-3, 1.0, xs)
    ym, ys = T.mean(axis=0), T.std(axis=0)
    ys = np.where(ys < 1e-3, 1.0, ys)
    return xm, xs, ym, ys


def make_blob(w: np.ndarray, xm, xs, ym, ys) -> np.ndarray:
    return np.concatenate([np.asarray(w, np.float32).ravel(), np.asarray(xm, np.float32), np.asarray(xs, np.float32),
                           np.asarray(ym, np.float32), np.asarray(ys, np.float32)]).astype(np.float32)


def init_weights(seed: int) -> np.ndarray:
    """Fan-in scaled uniform initialisation from the counter-based generator."""
    w = np.zeros(4866, dtype=np.float64)
    w[0:512] = wl.uniform(seed, 1, 512, -1.0, 1.0) * math.sqrt(6.0 / 8)
    w[576:4672] = wl.uniform(seed, 2, 4096, -1.0, 1.0) * math.sqrt(6.0 / 64)
    w[4736:4864] = wl.uniform(seed, 3, 128, -1.0, 1.0) * math.sqrt(6.0 / 64) * 0.1
    return w.astype(np.float32)


# --------------------------------------------------------------------------------------
# GPU steps (library calls)
# --------------------------------------------------------------------------------------
def collect_traces(solver, problems: list, chunk: int = 128) -> list:
    """Solve problems with the paper's controller (batched launches) and return their records."""
    import torch
    from . import phipm as pm
    solver.set_controller(0)
    solver.trace_enable(1 << 20)
    records = []
    for c0 in range(0, len(problems), chunk):
        part = problems[c0:c0 + chunk]
        ops = [pm.DeviceOperator(p_.op) for p_ in part]
        bs = [[torch.as_tensor(x).cuda() for x in p_.b] for p_ in part]
        solver.solve_batched([p_.t_end for p_ in part], ops, bs, [p_.tol for p_ in part], [p_.symm for p_ in part])
        for r in solver.trace_read():
            r = dict(r)
            r["problem"] += c0
            records.append(r)
    solver.trace_enable(0)
    return records


def train(solver, X: np.ndarray, T: np.ndarray, iters: int = 3000, lr: float = 3e-3, seed: int = 11):
    """Full-batch Adam on standardised data through phipm_mlp_train; returns (blob, losses)."""
    import torch
    xm, xs, ym, ys = standardise(X, T)
    Xn = torch.as_tensor(((X - xm) / xs).astype(np.float32)).cuda().contiguous()
    Tn = torch.as_tensor(((T - ym) / ys).astype(np.float32)).cuda().contiguous()
    w = torch.as_tensor(init_weights(seed)).cuda()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    losses = solver.mlp_train(w, m, v, Xn, Tn, iters, 0, lr)
    return make_blob(w.cpu().numpy(), xm, xs, ym, ys), losses
