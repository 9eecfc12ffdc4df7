"""Benchmark of the phipm hot path on GB300: one JSON line on rank 0.

A step is one full solve u(t_end) = sum_k t^k phi_k(tA) b_k (Sec. 3, Algorithm 3)
of the FP64 nonsymmetric workload: 2D convection-diffusion, 512 x 512 grid
(n = 262144), diffusion 1, velocity (50, 50), central differences, CSR float64 /
int32, p = 4, b_k ~ N(0,1) (seeded), t_end = 1e-3, Tol = 1e-8.

  value      solves/s over all ranks, inputs resident in HBM, device-timed with
             CUDA events, L2 flushed (256 MiB write) between timed solves
  e2e        the same through phipm_solve_host: H2D of A and b from pinned host
             memory, the solve, D2H of u, every step
  roofline   the solver kernel's algorithmic bytes (SpMV + Arnoldi per-step
             model: two passes over the basis per step) / its event-timed
             duration, against the measured copy bandwidth
  cpu_baseline  the FP64 CPU oracle (as it stands) timed on the host, one
             full solve of the same seeded inputs; its result also checks parity

--impl reference times the oracle alone (the method's reference implementation
on the host cores) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "convdiff2d_512": dict(metric_cfg="FP64 nonsymmetric (Arnoldi) convection-diffusion 512x512 CSR, p=4",
                           precision="f64", extras=["f64pair"]),
    "laplacian2d_32": dict(metric_cfg="plain FP64 32x32 Laplacian stencil, p=3 (Lanczos)", precision="f64",
                           extras=["f64pair"]),
    "laplacian3d_128": dict(metric_cfg="FP32-basis 128^3 Laplacian stencil, p=2, tol 1e-5", precision="f32"),
    "heston_100x51": dict(metric_cfg="Heston PDE (Sec. 4.1), 100x51 grid, n 5100, u' = Au + b_1, T = 1, tol 1e-4",
                          precision="f64", extras=["f64pair"]),
    "ninepoint30_phi4": dict(metric_cfg="nine-point 30x30 matrix (n 900, nnz 7,744), sum of t^k phi_k(tA) 1, "
                                        "k <= 4, t = 2, tol 2^-26 (Sec. 4.2, Experiment 2), phipm", precision="f64",
                             extras=["f64pair"]),
    "ninepoint30_phi4_phip": dict(metric_cfg="the same problem with the fixed-dimension variant phip (m = 30)",
                                  precision="f64", extras=["f64pair"], params=dict(controller=2, m_init=30)),
    "batched_convdiff_256": dict(metric_cfg="256 independent convection-diffusion problems, sides U{64..256}, "
                                            "p U{1..4}, tol 1e-8, one persistent launch replayed as a CUDA graph",
                                 precision="f64", batched=True, extras=["f64pair", "f32"]),
    "batched_convdiff_256_f32": dict(metric_cfg="the same 256 problems with an FP32 Krylov basis, tol 1e-5",
                                     precision="f32", batched=True, tol=1e-5),
    "peclet_128_1024_learned": dict(metric_cfg="1024 held-out convection-diffusion 128x128 problems, Peclet "
                                               "log-uniform [1,1e3], tol 1e-8, learned (tau, m) controller",
                                    precision="f64", batched=True, learned=True, extras=["f64pair"]),
}
DTYPES = {"f64": "f64", "f32": "f32 basis (FP64 coefficients, H, expm, eps, u)",
          "f64pair": "f32x2 float pairs on the FP32 pipe (FP64-class; FP64 w-recurrence, H, expm, eps, u)"}
# tolerance of each precision form when it runs as another form of a workload
EXTRA_TOL = {"f32": 1e-5}
KERNEL_ELEM = {"f64": "<double>", "f32": "<float>", "f64pair": "<df32>"}
# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz (maximum SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
METRIC = "solves/s at rel.err<=1e-8 vs FP64 oracle; SpMV+Arnoldi HBM GB/s vs peak"
PEAK_FALLBACK = 6800.0


def make_batch(name: str, first: int = 0, count: int | None = None) -> list:
    """Problems [first, first+count) of a batched workload (each depends on its own seed only)."""
    from paper_0907_4631_gb300 import workloads as wl
    spec = WORKLOADS[name]
    if name.startswith("batched_convdiff_256"):
        total = 256
        cnt = total - first if count is None else count
        probs = wl.batched_convdiff_problems(count=cnt, seed0=4000 + first)
    elif name == "peclet_128_1024_learned":
        total = 1024
        cnt = total - first if count is None else count
        probs = wl.peclet_convdiff_problems(count=cnt, seed0=5000 + first)
    else:
        raise ValueError(name)
    if "tol" in spec:
        for pr in probs:
            pr.tol = spec["tol"]
    return probs


def make_problem(name: str):
    from paper_0907_4631_gb300 import workloads as wl
    if name == "convdiff2d_512":
        return wl.convdiff_2d_problem()
    if name == "laplacian2d_32":
        return wl.laplacian_2d_problem()
    if name == "laplacian3d_128":
        return wl.laplacian_3d_problem()
    if name == "heston_100x51":
        return wl.heston_problem()
    if name.startswith("ninepoint30_phi4"):
        return wl.nine_point_phi_sum_problem(30)
    raise ValueError(name)


def oracle_params(name: str) -> dict:
    """The oracle's parameters for a workload's controller (phip: adapt_m off, m = m_init)."""
    prm = WORKLOADS[name].get("params", {})
    if prm.get("controller") == 2:
        return dict(adapt_m=False, m_init=prm.get("m_init", 10))
    return {}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK, "fallback"


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (replicas: whole-job throughput is bounded by it)."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, total_ms: float) -> float:
    """Units per second of the whole job: every rank processes units_per_rank in total_ms."""
    return world * units_per_rank / (total_ms / 1e3)


def algorithmic_bytes(pr, stats, precision) -> float:
    """SpMV + Arnoldi bytes of one solve (per-step model).

    An Arnoldi step j (lagged Gram-Schmidt) reads the j basis vectors twice (the
    dot pass and the fused update), summed as 2 s n gs_vectors; it reads the
    candidate and A times the candidate twice and writes the new basis vector
    and the next candidate (6 s n), and runs one SpMV (CSR: 12 nnz + 4 (n+1) +
    2 s n for the x read and the y write; stencil: 2 s n).  A Lanczos step reads
    v_j for the dot, v_{j-1}, v_j and y for the update and writes y, reads y for
    the norm, and writes the next basis vector."""
    n = pr.n
    s = 4 if precision == "f32" else 8
    if hasattr(pr.op, "rowptr"):
        spmv = 12 * pr.op.nnz + 4 * (n + 1) + 2 * s * n
    else:
        spmv = 2 * s * n
    kry = stats["krylov_steps"]
    gs = stats["gs_vectors"]
    if gs == 0:   # Lanczos
        per_step = spmv + s * n * (2 + 4) + s * n
        return kry * per_step
    return 2.0 * s * n * gs + kry * (spmv + 6.0 * s * n)


def fp64_flops(pr, stats) -> float:
    """FP64 flops of one solve's Krylov phase with the IEEE FP64 basis: an Arnoldi step j
    takes j n fused multiply-adds in the dot pass (V^T w) and j n in the fused update
    (w - V b), twice that when it also forms the candidate's second projection (V^T z,
    z - V a; counted by reorth_vectors), plus one SpMV (nnz) and the finishing scalings
    (4 n); a Lanczos step takes 3 n + 2 n (dot, three-term update) + nnz + 2 n (norm,
    scaling)."""
    n = pr.n
    nnz = pr.op.nnz if hasattr(pr.op, "rowptr") else pr.op.nnz()
    kry, gs = stats["krylov_steps"], stats["gs_vectors"]
    if gs == 0:
        return 2.0 * kry * (nnz + 7.0 * n)
    reorth = stats.get("reorth_vectors", gs)
    return 2.0 * (2.0 * n * (gs + reorth) + kry * (nnz + 4.0 * n))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_oracle_subprocess(workload: str, horizon: float, save_u: str | None) -> tuple:
    """Time the CPU oracle on the same seeded inputs in a fresh single-threaded process."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
from bench import make_problem, oracle_params
from oracle import phipm_oracle as O
pr = make_problem({workload!r})
t0 = time.perf_counter()
u, st = O.phipm(pr.t_end * {horizon!r}, pr.op, pr.b, pr.tol, pr.symm, oracle_params({workload!r}))
dt = time.perf_counter() - t0
if {save_u!r}:
    np.save({save_u!r}, u)
print(json.dumps(dict(seconds=dt, steps=st.steps, rejects=st.rejects)))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def _oracle_batch_worker(job):
    """One oracle solve of problem idx of a batched workload (in a spawned process)."""
    import time as _t
    import numpy as _np
    from oracle import phipm_oracle as O
    workload, idx, path = job
    pr = make_batch(workload, idx, 1)[0]
    t0 = _t.perf_counter()
    u, st = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, pr.symm)
    dt = _t.perf_counter() - t0
    _np.save(path, u)
    return dt, st.steps, st.rejects


def run_oracle_pool(workload: str, indices: list, tmpdir: str) -> tuple:
    """Oracle solves of the given problems, spread over the host cores by a spawned
    process pool (single-threaded BLAS each).  Returns (wall seconds, cores, per-problem u paths)."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    cores = max(1, min(len(indices), os.cpu_count() or 1))
    paths = [os.path.join(tmpdir, f"u_{i}.npy") for i in indices]
    ctx = mp.get_context("spawn")
    saved = os.environ.get("CUDA_VISIBLE_DEVICES")
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    try:
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_batch_worker, [(workload, 0, os.path.join(tmpdir, "warm.npy"))] * cores, chunksize=1)
            t0 = time.perf_counter()
            res = pool.map(_oracle_batch_worker, [(workload, i, pth) for i, pth in zip(indices, paths)], chunksize=1)
            wall = time.perf_counter() - t0
    finally:
        if saved is None:
            del os.environ["CUDA_VISIBLE_DEVICES"]
        else:
            os.environ["CUDA_VISIBLE_DEVICES"] = saved
    return wall, cores, paths, res


def traffic_from_profiles(kernel: str, workload: str):
    """dram bytes per launch from a committed ncu summary, if it matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
        ent = d[f"{kernel}@{workload}"]
        from paper_0907_4631_gb300 import build as b
        if ent.get("source_hash") != b.source_hash():
            return None
        return float(ent["dram_bytes_per_launch"])
    except Exception:
        return None


def reference_arm_batched(args, world):
    """The oracle on bounded samples of a batched workload: each step solves one problem
    per host core (a window moving through the batch), spread over spawned processes."""
    count = len(make_batch(args.workload))
    cores = os.cpu_count() or 1
    secs, solved = [], 0
    with tempfile.TemporaryDirectory() as td:
        for k in range(args.warmup + args.steps):
            idx = [((k * cores + j) * 7) % count for j in range(cores)]
            wall, used, _, _ = run_oracle_pool(args.workload, idx, td)
            if k >= args.warmup:
                secs.append(wall)
                solved += len(idx)
    total = sum(secs)
    value = solved / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded counter-based generator)",
        "config": {"workload": args.workload, "problems": count},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": min(cores, count), "kind": "oracle",
                         "sample": f"per step {cores} problems of the batch, one FP64 oracle solve each over "
                                   f"spawned processes (value = problems / seconds)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reference_arm(args, world, rank):
    if rank != 0:
        return
    if WORKLOADS[args.workload].get("batched"):
        reference_arm_batched(args, world)
        return
    pr = make_problem(args.workload)
    # each step: the oracle over a fraction f of [0, t_end], so the run stays within minutes
    f = min(1.0, 6.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        run_oracle_subprocess(args.workload, f, None)
    secs = []
    for _ in range(args.steps):
        secs.append(run_oracle_subprocess(args.workload, f, None)["seconds"])
    total = sum(secs)
    value = args.steps * f / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded counter-based generator)",
        "config": {"workload": args.workload, "n": pr.n, "p": pr.p, "t_end": pr.t_end, "tol": pr.tol},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"FP64 numpy/scipy oracle over the first {f:.3f} of [0, t_end] per step "
                                   f"(value = fraction of a solve / seconds)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_batch(batch, stream, flush, steps, packed=None):
    """Event-timed repeats of one batched solve; with packed, each repeat also uploads the
    inputs from pinned host memory and downloads every u (the end-to-end leg)."""
    import torch
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if packed is not None:
            packed.upload(stream)
        batch.run(stream)
        if packed is not None:
            packed.download(stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def run_batched(args, world, rank, local):
    import numpy as np
    import torch
    from paper_0907_4631_gb300 import phipm as pm
    spec = WORKLOADS[args.workload]
    prec = spec["precision"]
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    probs = make_batch(args.workload, 0, args.count if args.count > 0 else None)
    count = len(probs)
    solver = pm.Phipm(prec)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    learned = None
    if spec.get("learned"):
        from paper_0907_4631_gb300 import learned as L
        t0 = time.perf_counter()
        tr = L.training_problems(count=768, seed0=7000)
        traces = L.collect_traces(solver, tr)
        X, T = L.examples_from_traces(traces)
        blob, losses = L.train(solver, X, T, iters=3000, lr=3e-3)
        solver.set_controller_weights(blob)
        learned = {"training_problems": len(tr), "examples": int(X.shape[0]), "adam_iters": 3000,
                   "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                   "train_seconds": time.perf_counter() - t0}
    pk = PackedBatch(probs)
    batch = solver.batch([pr.t_end for pr in probs], pk.ops, pk.bs, [pr.tol for pr in probs],
                         [pr.symm for pr in probs], outs=pk.outs)

    tune = None
    if not args.no_autotune:     # untimed: picks the cluster size K for this batch class
        tune = batch.autotune(stream)

    def measure(controller):
        solver.set_controller(controller)
        for _ in range(args.warmup):
            batch.run(stream)
        torch.cuda.synchronize()
        return time_batch(batch, stream, flush, args.steps), batch.stats()

    plain = every = None
    if learned is not None:
        # the learned controller that proposes every step, with its own network (reported;
        # the headline keeps the first-step proposal, measured faster)
        X3, T3 = L.examples_every_step(traces)
        blob3, losses3 = L.train(solver, X3, T3, iters=3000, lr=3e-3)
        solver.set_controller_weights(blob3)
        max_steps = solver.params.max_steps
        solver.params.max_steps = 2000       # bounds the run if a trained network stalls a solve
        et_, est = measure(3)
        solver.params.max_steps = max_steps
        every = {"value": world * count * args.steps / (sum(et_) / 1e3), "unit": "solves/s",
                 "problems_not_ok": int(sum(1 for x in batch.statuses() if x != pm.OK)),
                 "examples": int(X3.shape[0]), "loss_last": float(losses3[-1]),
                 "rejects": int(sum(x["rejects"] for x in est)), "steps": int(sum(x["steps"] for x in est)),
                 "matvecs": int(sum(x["matvecs"] for x in est)),
                 "gs_vectors": int(sum(x["gs_vectors"] for x in est))}
        solver.set_controller_weights(blob)
        pt, pst = measure(0)
        plain = {"value": world * count * args.steps / (sum(pt) / 1e3), "unit": "solves/s",
                 "rejects": int(sum(x["rejects"] for x in pst)), "steps": int(sum(x["steps"] for x in pst)),
                 "matvecs": int(sum(x["matvecs"] for x in pst)),
                 "krylov_steps": int(sum(x["krylov_steps"] for x in pst)),
                 "gs_vectors": int(sum(x["gs_vectors"] for x in pst))}
        u_plain = [u.cpu().numpy() for u in pk.outs]
    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        batch.run(stream)
    solver.set_controller(1 if learned is not None else 0)
    for _ in range(args.warmup):
        batch.run(stream)
    torch.cuda.synchronize()
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times = time_batch(batch, stream, flush, args.steps)
    stats = batch.stats()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(times), dist, "cuda")
    value = replica_throughput(count * args.steps, world, total_ms)
    kernel_ms = stats[0]["kernel_ms"]
    u_gpu = [u.cpu().numpy() for u in pk.outs]

    # end to end: inputs uploaded from one pinned host buffer, every u downloaded, each step
    e2e = None
    if not args.no_e2e:
        et = time_batch(batch, stream, flush, args.steps, packed=pk)
        tot = max_over_ranks(sum(et), dist, "cuda")
        e2e = {"value": replica_throughput(count * args.steps, world, tot), "unit": "solves/s",
               "h2d_bytes_per_step": int(pk.in_bytes), "d2h_bytes_per_step": int(pk.out_bytes)}

    # the plain FP64 GPU solver, one problem per call, on an evenly spaced sample
    sample = list(range(0, count, max(1, count // 32)))
    f64 = pm.Phipm("f64")
    for i in sample[:3]:
        f64.solve(probs[i].t_end, pk.ops[i], pk.bs[i], probs[i].tol, probs[i].symm)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in sample:
        f64.solve(probs[i].t_end, pk.ops[i], pk.bs[i], probs[i].tol, probs[i].symm)
    e1.record(stream)
    e1.synchronize()
    plain_f64 = {"value": len(sample) / (e0.elapsed_time(e1) / 1e3), "unit": "solves/s",
                 "sample": f"{len(sample)} problems (every {max(1, count // 32)}th), one phipm_solve each, "
                           f"FP64 basis, same tol"}

    team = solver.last_batched_team()
    roofline = roofline_batched(probs, stats, prec, kernel_ms, team, args.workload)

    # the other precision modes of the same batch, timed the same way (not the headline)
    extras, u_extra = {}, {}
    for xp in spec.get("extras", []):
        sx = pm.Phipm(xp)
        if learned is not None:
            sx.set_controller_weights(blob)
            sx.set_controller(1)
        tolx = EXTRA_TOL.get(xp)
        outs_x = [torch.empty_like(x) for x in pk.outs]
        bx = sx.batch([pr.t_end for pr in probs], pk.ops, pk.bs, [tolx or pr.tol for pr in probs],
                      [pr.symm for pr in probs], outs=outs_x)
        if not args.no_autotune:
            bx.autotune(stream)
        for _ in range(args.warmup):
            bx.run(stream)
        torch.cuda.synchronize()
        xt = time_batch(bx, stream, flush, args.steps)
        xst = bx.stats()
        xtot = max_over_ranks(sum(xt), dist, "cuda")
        tx = sx.last_batched_team()
        extras[xp] = {"value": replica_throughput(count * args.steps, world, xtot), "unit": "solves/s",
                      "ms_per_step": xtot / args.steps, "dtype": DTYPES[xp], "tol": tolx or probs[0].tol,
                      "team": tx,
                      "solver_stats": {k: int(sum(x[k] for x in xst)) for k in ("steps", "rejects", "krylov_steps",
                                                                                 "gs_vectors", "reorth_vectors")},
                      "roofline": roofline_batched(probs, xst, xp, xst[0]["kernel_ms"], tx, args.workload)}
        u_extra[xp] = [x.cpu().numpy() for x in outs_x]
        del bx
        sx.close()
    sizes = [pr.n for pr in probs]
    convert = prec != "f64"
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec],
        "data": "synthetic (seeded counter-based generator; same inputs as the oracle)",
        "config": {"workload": args.workload, "problems": count, "n_min": min(sizes), "n_max": max(sizes),
                   "n_total": int(sum(sizes)), "tol": probs[0].tol,
                   "l2": "flushed between timed batches (256 MiB write)",
                   "launch": "one persistent queue kernel per batch, replayed from a captured CUDA graph",
                   "team": team, "autotune_ms": {str(k): round(ms, 3) for k, ms in tune} if tune else None,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "solver_stats": {k: int(sum(x[k] for x in stats)) for k in ("steps", "rejects", "matvecs", "expms",
                                                                     "krylov_steps", "gs_vectors",
                                                                     "reorth_vectors")},
        "gpu_launches": args.steps * (2 if convert else 1),
        "roofline": roofline,
        "clocks": clocks,
        "plain_fp64_gpu_solver": plain_f64,
    }
    if extras:
        line["other_precisions"] = extras
    if learned is not None:
        line["learned"] = learned
        line["plain_controller"] = plain
        line["learned_every_step_controller"] = every
        line["learned_first_step_counters"] = {k: int(sum(x[k] for x in stats))
                                               for k in ("rejects", "steps", "matvecs", "gs_vectors")}
        line["plain_vs_learned_max_rel_diff"] = float(max(
            np.linalg.norm(a - b_) / np.linalg.norm(b_) for a, b_ in zip(u_gpu, u_plain)))
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        csample = list(range(0, count, max(1, count // 48)))[:48]
        with tempfile.TemporaryDirectory() as td:
            wall, cores, paths, res = run_oracle_pool(args.workload, csample, td)
            u_ref = {i: np.load(pth) for i, pth in zip(csample, paths)}

        def rel_errs(us):
            return [float(np.linalg.norm(us[i] - ur) / np.linalg.norm(ur)) for i, ur in u_ref.items()]
        errs = rel_errs(u_gpu)
        line["cpu_baseline"] = {"value": len(csample) / wall, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                "sample": f"{len(csample)} of the {count} problems (evenly spaced), one FP64 "
                                          f"oracle solve each, spread over {cores} spawned processes"}
        line["rel_err_vs_oracle"] = {"max": max(errs), "median": statistics.median(errs), "problems": len(errs)}
        for xp, ux in u_extra.items():       # against the oracle at the headline's tolerance
            xe = rel_errs(ux)
            extras[xp]["rel_err_vs_oracle"] = {"max": max(xe), "median": statistics.median(xe), "problems": len(xe)}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def roofline_batched(probs, stats, prec, kernel_ms, team, workload) -> dict:
    """Algorithmic SpMV + Arnoldi bytes of every problem of the batch over the batched
    kernel's event-timed duration, against the measured copy bandwidth."""
    peak, peak_kind = measured_peaks()
    abytes = sum(algorithmic_bytes(pr, st, prec) for pr, st in zip(probs, stats))
    achieved = abytes / (kernel_ms / 1e3) / 1e9
    kernel_name = ("k_solve_cluster" if team >= 2 else "k_solve_queue") + KERNEL_ELEM[prec]
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic_from_profiles(kernel_name, workload), "peak_kind": peak_kind, "kernel": kernel_name,
           "algorithmic_bytes_per_launch": abytes, "kernel_ms": kernel_ms}
    if prec == "f64":
        fl = sum(fp64_flops(pr, st) for pr, st in zip(probs, stats))
        out["fp64_pipe"] = {"achieved": fl / (kernel_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": fl / (kernel_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "flops_per_launch": fl,
                            "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"}
    return out


class PackedBatch:
    """All inputs of a batch in one pinned host buffer and one device buffer (256-byte
    aligned arrays), so the end-to-end leg moves them with one copy each way."""

    def __init__(self, probs):
        import numpy as np
        import torch
        from paper_0907_4631_gb300 import phipm as pm
        lay, off = [], 0

        def take(nbytes):
            nonlocal off
            o = off
            off += (nbytes + 255) // 256 * 256
            return o
        for pr in probs:
            ent = {"b": [take(8 * pr.n) for _ in pr.b]}
            if hasattr(pr.op, "rowptr"):
                ent["csr"] = (take(4 * (pr.n + 1)), take(4 * pr.op.nnz), take(8 * pr.op.nnz))
            lay.append(ent)
        in_bytes = off
        self.u_off = [take(8 * pr.n) for pr in probs]
        self.in_bytes, self.out_bytes = in_bytes, off - in_bytes
        host = np.zeros(off, dtype=np.uint8)
        for pr, ent in zip(probs, lay):
            for o, x in zip(ent["b"], pr.b):
                host[o:o + 8 * pr.n] = np.ascontiguousarray(x, dtype=np.float64).view(np.uint8)
            if "csr" in ent:
                for o, x, dt in zip(ent["csr"], (pr.op.rowptr, pr.op.colind, pr.op.values),
                                    (np.int32, np.int32, np.float64)):
                    a = np.ascontiguousarray(x, dtype=dt).view(np.uint8)
                    host[o:o + a.size] = a
        self.host = torch.from_numpy(host).pin_memory()
        self.dev = torch.empty(off, dtype=torch.uint8, device="cuda")
        self.dev.copy_(self.host)

        def view(o, count, dt):
            return self.dev[o:o + count * torch.empty((), dtype=dt).element_size()].view(dt)
        self.ops, self.bs = [], []
        for pr, ent in zip(probs, lay):
            self.bs.append([view(o, pr.n, torch.float64) for o in ent["b"]])
            arrays = None
            if "csr" in ent:
                arrays = (view(ent["csr"][0], pr.n + 1, torch.int32), view(ent["csr"][1], pr.op.nnz, torch.int32),
                          view(ent["csr"][2], pr.op.nnz, torch.float64))
            self.ops.append(pm.DeviceOperator(pr.op, arrays=arrays))
        self.outs = [view(o, pr.n, torch.float64) for o, pr in zip(self.u_off, probs)]
        self.host_out = torch.empty(self.out_bytes, dtype=torch.uint8).pin_memory()

    def upload(self, stream):
        with torch_stream(stream):
            self.dev[:self.in_bytes].copy_(self.host[:self.in_bytes], non_blocking=True)

    def download(self, stream):
        with torch_stream(stream):
            self.host_out.copy_(self.dev[self.in_bytes:], non_blocking=True)

    def u_host(self, i, n):
        o = self.u_off[i] - self.in_bytes
        return self.host_out[o:o + 8 * n].numpy().view("<f8")


def torch_stream(stream):
    import torch
    return torch.cuda.stream(stream)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="convdiff2d_512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default team size (no phipm_autotune)")
    ap.add_argument("--count", type=int, default=0, help="batched workloads: only the first COUNT problems")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    if WORKLOADS[args.workload].get("batched"):
        run_batched(args, world, rank, local)
        return

    import numpy as np
    import torch
    from paper_0907_4631_gb300 import phipm as pm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    pr = make_problem(args.workload)
    spec = WORKLOADS[args.workload]
    prec = spec["precision"]
    A = pm.DeviceOperator(pr.op)
    b = [torch.as_tensor(x).cuda() for x in pr.b]
    u = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    is_csr = hasattr(pr.op, "rowptr")

    solver = pm.Phipm(prec, **spec.get("params", {}))
    tune = None
    if not args.no_autotune:     # untimed: picks the team size for this size class
        tune = solver.autotune(pr.t_end, A, b, pr.tol, pr.symm, out=u)
    team = solver.team_for(0 if is_csr else 1, pr.n)
    for _ in range(args.warmup):
        solver.solve(pr.t_end, A, b, pr.tol, pr.symm, out=u)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, kms, stats = time_solves(solver, pr, A, b, u, flush, stream, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(times), dist, "cuda")
    value = replica_throughput(args.steps, world, total_ms)
    u_gpu = u.cpu().numpy()

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        hostA = pm.HostOperator(pr.op)
        pinned = []
        if is_csr:
            for arr in (hostA.rowptr, hostA.colind, hostA.values):
                pt = torch.from_numpy(arr).pin_memory()
                pinned.append(pt)
            hostA.c.csr.rowptr, hostA.c.csr.colind, hostA.c.csr.values = [x.data_ptr() for x in pinned]
        bh = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in pr.b]
        uh = torch.empty(pr.n, dtype=torch.float64).pin_memory()
        for _ in range(2):
            solver.solve_host(pr.t_end, hostA, bh, pr.tol, pr.symm, out=uh)
        h2d = sum(x.numel() * x.element_size() for x in bh + pinned)
        d2h = uh.numel() * uh.element_size()
        et = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve_host(pr.t_end, hostA, bh, pr.tol, pr.symm, out=uh)
            e1.record(stream)
            e1.synchronize()
            et.append(e0.elapsed_time(e1))
        tot = max_over_ranks(sum(et), dist, "cuda")
        e2e = {"value": replica_throughput(args.steps, world, tot), "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    roofline = roofline_single(pr, stats, prec, statistics.mean(kms), team, args.workload)

    # the other precision modes of the same workload, timed the same way (not the headline)
    extras, u_extra = {}, {}
    for xp in spec.get("extras", []):
        sx = pm.Phipm(xp, **spec.get("params", {}))
        ux = torch.empty(pr.n, dtype=torch.float64, device="cuda")
        if not args.no_autotune:
            sx.autotune(pr.t_end, A, b, pr.tol, pr.symm, out=ux)
        tx = sx.team_for(0 if is_csr else 1, pr.n)
        for _ in range(args.warmup):
            sx.solve(pr.t_end, A, b, pr.tol, pr.symm, out=ux)
        torch.cuda.synchronize()
        xt, xk, xs = time_solves(sx, pr, A, b, ux, flush, stream, args.steps)
        xtot = max_over_ranks(sum(xt), dist, "cuda")
        extras[xp] = {"value": replica_throughput(args.steps, world, xtot), "unit": "solves/s",
                      "ms_per_step": xtot / args.steps, "dtype": DTYPES[xp], "team": tx,
                      "solver_stats": {k: xs[k] for k in ("steps", "rejects", "krylov_steps", "gs_vectors",
                                                           "reorth_vectors")},
                      "roofline": roofline_single(pr, xs, xp, statistics.mean(xk), tx, args.workload)}
        u_extra[xp] = ux.cpu().numpy()
        sx.close()

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec],
        "data": "synthetic (seeded counter-based generator; same inputs as the oracle)",
        "config": {"workload": args.workload, "n": pr.n, "nnz": int(pr.op.nnz if is_csr else pr.op.nnz()),
                   "p": pr.p, "t_end": pr.t_end, "tol": pr.tol, "l2": "flushed between timed solves (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "team": team, "autotune_ms": {str(t): round(ms, 3) for t, ms in tune} if tune else None},
        "solver_stats": {k: stats[k] for k in ("steps", "rejects", "matvecs", "expms", "krylov_steps", "gs_vectors",
                                                "reorth_vectors")},
        "gpu_launches": args.steps * (2 if (prec != "f64" and is_csr) else 1),
        "roofline": roofline,
        "clocks": clocks,
    }
    if extras:
        line["other_precisions"] = extras
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        tmpu = tempfile.mktemp(suffix=".npy")
        r = run_oracle_subprocess(args.workload, 1.0, tmpu)
        u_ref = np.load(tmpu)
        os.unlink(tmpu)
        line["cpu_baseline"] = {"value": 1.0 / r["seconds"], "unit": "solves/s", "cores": 1, "kind": "oracle",
                                "sample": "one full solve of the same seeded workload (FP64 numpy/scipy oracle, "
                                          "single-threaded BLAS)"}
        line["rel_err_vs_oracle"] = float(np.linalg.norm(u_gpu - u_ref) / np.linalg.norm(u_ref))
        for xp, ux in u_extra.items():
            extras[xp]["rel_err_vs_oracle"] = float(np.linalg.norm(ux - u_ref) / np.linalg.norm(u_ref))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def time_solves(solver, pr, A, b, u, flush, stream, steps):
    """Event-timed full solves on resident inputs, L2 flushed before each; returns the
    per-solve times (ms), the solver kernel's own times (ms) and the last solve's stats."""
    import torch
    times, kms, stats = [], [], None
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, stats, _ = solver.solve(pr.t_end, A, b, pr.tol, pr.symm, out=u)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        kms.append(stats["kernel_ms"])
    return times, kms, stats


def roofline_single(pr, stats, prec, kernel_ms, team, workload) -> dict:
    """The solver kernel's algorithmic SpMV + Arnoldi bytes over its event-timed duration,
    against the measured copy bandwidth; for the IEEE FP64 basis also its FP64 arithmetic
    (Gram-Schmidt and SpMV fused multiply-adds) against the FP64 pipe's peak."""
    peak, peak_kind = measured_peaks()
    abytes = algorithmic_bytes(pr, stats, prec)
    achieved = abytes / (kernel_ms / 1e3) / 1e9
    kernel_name = ("k_solve_grid" if team >= 9 else "k_solve_cluster" if team >= 2 else "k_solve_queue") + \
        KERNEL_ELEM[prec]
    traffic = traffic_from_profiles(kernel_name, workload)
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel_name,
           "algorithmic_bytes_per_launch": abytes, "kernel_ms": kernel_ms}
    if prec == "f64":
        fl = fp64_flops(pr, stats)
        out["fp64_pipe"] = {"achieved": fl / (kernel_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": fl / (kernel_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                            "flops_per_launch": fl, "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"}
    return out


if __name__ == "__main__":
    main()
