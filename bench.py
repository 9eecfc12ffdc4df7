"""Benchmark of the phipm hot path on GB300: one JSON line on rank 0.

A step is one full solve u(t_end) = sum_k t^k phi_k(tA) b_k (Sec. 3, Algorithm 3)
of the FP64 nonsymmetric workload: 2D convection-diffusion, 512 x 512 grid
(n = 262144), diffusion 1, velocity (50, 50), central differences, CSR float64 /
int32, p = 4, b_k ~ N(0,1) (seeded), t_end = 1e-3, Tol = 1e-8.

  value      solves/s over all ranks, inputs resident in HBM, device-timed with
             CUDA events, L2 flushed (256 MiB write) between timed solves
  e2e        the same through phipm_solve_host: H2D of A and b from pinned host
             memory, the solve, D2H of u, every step
  roofline   the solver kernel's algorithmic HBM bytes (SpMV + Arnoldi/CGS2
             per-step model) / its event-timed duration, against the measured
             copy bandwidth
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
                           precision="f64pair"),
    "laplacian2d_32": dict(metric_cfg="plain FP64 32x32 Laplacian stencil, p=3 (Lanczos)", precision="f64pair"),
    "laplacian3d_128": dict(metric_cfg="FP32-basis 128^3 Laplacian stencil, p=2, tol 1e-5", precision="f32"),
}
DTYPES = {"f64": "f64", "f32": "f32 basis (FP64 coefficients, H, expm, eps, u)",
          "f64pair": "f32x2 float pairs on the FP32 pipe (FP64-class; FP64 w-recurrence, H, expm, eps, u)"}
METRIC = "solves/s at rel.err<=1e-8 vs FP64 oracle; SpMV+Arnoldi HBM GB/s vs peak"
PEAK_FALLBACK = 6800.0


def make_problem(name: str):
    from paper_0907_4631_gb300 import workloads as wl
    if name == "convdiff2d_512":
        return wl.convdiff_2d_problem()
    if name == "laplacian2d_32":
        return wl.laplacian_2d_problem()
    if name == "laplacian3d_128":
        return wl.laplacian_3d_problem()
    raise ValueError(name)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK, "fallback"


def algorithmic_bytes(pr, stats, precision) -> float:
    """SpMV + Arnoldi bytes of one solve (per-step model).

    CGS2 step j touches j+1 basis vectors four times (two dot passes, two
    update passes): 4 (j+1) s n bytes, summed as 4 s n gs_vectors.  Each Krylov
    step also runs one SpMV (CSR: 12 nnz + 4 (n+1) + 2 s n for the x read and
    the y write; stencil: 2 s n) and writes the new basis vector (s n)."""
    n = pr.n
    s = 4 if precision == "f32" else 8
    if hasattr(pr.op, "rowptr"):
        spmv = 12 * pr.op.nnz + 4 * (n + 1) + 2 * s * n
    else:
        spmv = 2 * s * n
    kry = stats["krylov_steps"]
    gs = stats["gs_vectors"]
    if gs == 0:   # Lanczos: t_jj dot (v_j, y), three-term update (v_{j-1}, v_j, y r/w), norm
        per_step = spmv + s * n * (2 + 4) + s * n
        return kry * per_step
    return 4.0 * s * n * gs + kry * (spmv + s * n)


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
from bench import make_problem
from oracle import phipm_oracle as O
pr = make_problem({workload!r})
t0 = time.perf_counter()
u, st = O.phipm(pr.t_end * {horizon!r}, pr.op, pr.b, pr.tol, pr.symm)
dt = time.perf_counter() - t0
if {save_u!r}:
    np.save({save_u!r}, u)
print(json.dumps(dict(seconds=dt, steps=st.steps, rejects=st.rejects)))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


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


def reference_arm(args, world, rank):
    if rank != 0:
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="convdiff2d_512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, world, rank)
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
    solver = pm.Phipm(spec["precision"])
    A = pm.DeviceOperator(pr.op)
    b = [torch.as_tensor(x).cuda() for x in pr.b]
    u = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        solver.solve(pr.t_end, A, b, pr.tol, pr.symm, out=u)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, kms, stats = [], [], None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, stats, _ = solver.solve(pr.t_end, A, b, pr.tol, pr.symm, out=u)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        kms.append(stats["kernel_ms"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = sum(times)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)
    u_gpu = u.cpu().numpy()

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        hostA = pm.HostOperator(pr.op)
        pinned = []
        if hasattr(pr.op, "rowptr"):
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
        tot = sum(et)
        if dist:
            t = torch.tensor([tot], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot = float(t.item())
        e2e = {"value": world * args.steps / (tot / 1e3), "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    peak, peak_kind = measured_peaks()
    kernel_ms = statistics.mean(kms)
    abytes = algorithmic_bytes(pr, stats, spec["precision"])
    achieved = abytes / (kernel_ms / 1e3) / 1e9
    kernel_name = "k_solve_grid" if pr.n >= 16384 else "k_solve_queue"
    traffic = traffic_from_profiles(kernel_name, args.workload)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel_name,
                "algorithmic_bytes_per_launch": abytes, "kernel_ms": kernel_ms}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[spec["precision"]],
        "data": "synthetic (seeded counter-based generator; same inputs as the oracle)",
        "config": {"workload": args.workload, "n": pr.n, "nnz": int(pr.op.nnz if hasattr(pr.op, "rowptr") else pr.op.nnz()),
                   "p": pr.p, "t_end": pr.t_end, "tol": pr.tol, "l2": "flushed between timed solves (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "solver_stats": {k: stats[k] for k in ("steps", "rejects", "matvecs", "expms", "krylov_steps", "gs_vectors")},
        "gpu_launches": args.steps * (2 if (spec["precision"] == "f32" and hasattr(pr.op, "rowptr")) else 1),
        "roofline": roofline,
        "clocks": clocks,
    }
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
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
