#!/usr/bin/env python
"""Benchmark: time-to-1e-10 solve of the row-sampling SGS-preconditioned PCG method.

One step = one pass of the whole hot path over one problem: exact column scales, row
weights, prefix and Philox draws (lsq_sample_rows), sampled normal matrix and SGS operator
(lsq_build_precond), and PCG with true-residual restarts to a relative normal-equation
residual of 1e-10 (lsq_pcg_solve).  The workload is the ill-conditioned dense UDV problem:
A = U diag(sigma) V^T, 262144 x 512, sigma log-spaced from 1 to 1e-6 (kappa(A) = 1e6),
b = A x* + 1e-6 noise, s = ceil(4 n ln n) = 12777 draws, one forward + one backward sweep.
A (1 GiB in FP64) is larger than L2, so no flush is needed between steps.

Prints ONE JSON line on rank 0.  --impl reference times the CPU oracle (the method as
written, FP64, single thread) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-10 solve and HBM GB/s of Ap/Aᵀq/SGS; mixed/batched/adjoint vs FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["f64", "f32", "f32x2"], default="f32x2",
                    help="f64: FP64 values and arithmetic; f32: FP32 values + FP64 refinement; "
                         "f32x2: double-float pairs (FP32 units) + FP64 refinement")
    ap.add_argument("--m", type=int, default=262144)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--kappa", type=float, default=1e6)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--maxit", type=int, default=1000000)
    ap.add_argument("--inner-tol", type=float, default=0.0)
    ap.add_argument("--sweeps", type=int, default=1,
                    help="t of Alg. 3; 0 = the paper's comparison method (CG on the normalised A)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=10)
    ap.add_argument("--workload", choices=["udv", "gauss", "sparse", "graph", "adjoint", "batch", "tc", "sampling",
                                           "paper"],
                    default="udv",
                    help="udv: the timed benchmark; the others measure one other configuration alone")
    ap.add_argument("--device-loop", type=int, default=0,
                    help="CSR blocks of right-hand sides: 1 = one persistent launch per solve")
    ap.add_argument("--sweep-form", type=int, default=0,
                    help="one-column sparse sweeps: 0 by shape, 1 grid, 2 one CTA, 3 one cluster")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations and the FP64 comparison solve after the timed region")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# N > 1 runs N independent replicas (weak scaling): every rank solves its own problem with
# no data-path collective; the ranks meet only at the barriers around the timed region and
# in the max-over-ranks reduction of its duration.
def replica_seeds(rank):
    """Seeds of rank's problem: (matrix and right-hand side, row sampling)."""
    return 2 + rank, 1002 + rank


def max_over_ranks(ms, world, device):
    """The slowest rank's timed-region duration, known to every rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, ms):
    """Solves per second of the whole job: every rank's steps over the slowest rank's time."""
    return world * steps / (ms / 1e3)


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.stop_ev = threading.Event()
        self.th = None

    def _run(self):
        while not self.stop_ev.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self.stop_ev.wait(0.2)

    def start(self):
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def stop(self):
        self.stop_ev.set()
        if self.th:
            self.th.join(timeout=10)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 4 + k and r[4 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def make_problem(args, seed_base, device_matmul=True):
    import workloads as W
    mm = None
    if device_matmul:   # input generation only: the two large Cholesky-QR products on the device
        import torch
        mm = lambda X, Y: (torch.from_numpy(np.ascontiguousarray(X)).cuda()
                           @ torch.from_numpy(np.ascontiguousarray(Y)).cuda()).cpu().numpy()
    if args.workload == "gauss":   # Gaussian A (Sec. 5.1), b = A x* + 1e-3 noise
        mat = W.gaussian_dense(args.m, args.n, seed_base)
        xs, b = W.rhs_for(mat, 1, 1e-3, seed_base + 100)
        return mat, xs[0], b[0]
    mat = W.udv_dense(args.m, args.n, args.kappa, seed_base, matmul=mm)
    xs, b = W.rhs_for(mat, 1, 1e-6, seed_base + 100)
    return mat, xs[0], b[0]


def workload_name(args, m, n):
    if args.workload == "gauss":
        return f"gaussian_dense_{m}x{n}"
    return f"udv_dense_{m}x{n}_kappa{args.kappa:g}"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


# dram__bytes_read.sum + dram__bytes_write.sum over the algorithmic bytes of one k_pcg_dense
# launch, from the ncu capture of the 131072 x 512 UDV case (same kernel, same per-iteration
# pattern); reset to None whenever the kernel changes
TRAFFIC_RATIO = {"f32x2": 0.9995}


def pcg_algorithmic(args, m, n, info, es, es_res, es_op):
    """Algorithmic bytes and flops of one lsq_pcg_solve launch (one column)."""
    it = int(info.iters[0])
    outer = int(info.outer[0])
    a_bytes = m * n * es
    per_iter = a_bytes + n * n * es_op                  # one pass over A, one over the operator
    res_passes = 1 + max(outer - 1, 0) + 1              # h = Â^T b, restarts, final check
    byts = it * per_iter + res_passes * (m * n * es_res + 8 * m)
    flops = it * (4.0 * m * n + 2.0 * n * n) + res_passes * 4.0 * m * n
    return byts, flops


def cpu_oracle_sample(mat, b, seed, iters_gpu, cpu_iters):
    """Oracle (FP64, one thread) on a bounded sample of one solve: full setup (S1-S6) plus
    `cpu_iters` PCG iterations, extrapolated to the iteration count of a full solve."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    smp = oracle.Sample(mat, seed)
    Mo = oracle.SampledM(smp)
    t1 = time.perf_counter()
    oracle.pcg(smp.mat, smp.d, Mo, b=b, tol=1e-300, maxit=cpu_iters, max_outer=1)
    t2 = time.perf_counter()
    per_iter = (t2 - t1) / cpu_iters
    t_solve = (t1 - t0) + per_iter * max(iters_gpu, 1)
    return t_solve, (t1 - t0), per_iter


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    seed_base, seed = replica_seeds(0)
    mat, xs, b = make_problem(args, seed_base, device_matmul=False)
    times = []
    # iterations of a full FP64 solve of the default workload, as measured on the GPU's FP64
    # path (107,454 with the current kernel: the same textbook PCG as the oracle, another
    # summation order)
    iters_assumed = int(os.environ.get("LSQ_REF_ITERS", "107454"))
    for k in range(args.warmup + args.steps):
        t, ts, ti = cpu_oracle_sample(mat, b, seed, iters_assumed, args.cpu_iters)
        if k >= args.warmup:
            times.append(t)
    t = float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": 1.0 / t, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, args.m, args.n), "m": args.m, "n": args.n,
                       "kappa": args.kappa, "tol": args.tol, "sweeps": args.sweeps,
                       "s": math.ceil(4 * args.n * math.log(args.n)), "mode": args.mode,
                       "l2": "inputs larger than L2 (A is %.2f GB)" % (args.m * args.n * 8 / 1e9),
                       "parallelism": "replicas1"},
            "cpu_baseline": {"value": 1.0 / t, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"oracle setup (sampling, A_s^T A_s, SGS) on the full matrix + "
                                       f"{args.cpu_iters} PCG iterations per step, extrapolated to "
                                       f"{iters_assumed} iterations"},
            "e2e": {"value": 1.0 / t, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def gauss_config(steps=50, warmup=10, cpu=True):
    """The Gaussian dense configuration: A 4096 x 128 N(0,1), b = A x* + 1e-3 noise, FP64,
    s = ceil(4 n ln n), one forward + one backward sweep, tol 1e-10.  A step is sampling, the
    preconditioner and the solve; steps are timed with CUDA events on the stream (A, 4 MB,
    stays in L2, so the roofline fraction is of HBM bandwidth for a kernel that does not
    need it)."""
    import torch
    import workloads as W
    from paper_1806_02968_gb300 import api
    mat = W.gaussian_dense(4096, 128, 2)
    xs, b = W.rhs_for(mat, 1, 1e-3, 102)
    A = torch.from_numpy(mat["A"]).cuda()
    bd = torch.from_numpy(b[0]).cuda()
    Mx = api.Matrix(A)
    o = api.opts(seed=1002)
    stream = torch.cuda.current_stream()
    pcg = []

    def step():
        idx, p, d = api.lsq_sample_rows(Mx, o)
        P = api.lsq_build_precond(Mx, idx, p, d, o)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = api.lsq_pcg_solve(Mx, P, bd, o)
        e1.record(stream)
        return x, info, e0, e1
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    L0 = api.launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        x, info, e0, e1 = step()
        e1.synchronize()
        pcg.append(e0.elapsed_time(e1))
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    m, n = mat["A"].shape
    it = int(info.iters[0])
    byts = it * (m * n * 8 + n * n * 8) + (2 + max(int(info.outer[0]) - 1, 0)) * (m * n * 8 + 8 * m)
    pcg_s = float(np.mean(pcg)) / 1e3
    out = {"value": 1e3 / ms, "unit": "solves/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "dtype": "f64", "config": {"workload": "gaussian_dense_4096x128", "m": m, "n": n, "tol": 1e-10,
                                      "sweeps": 1, "s": int(info.s)},
           "iters": it, "relres_true": float(info.relres_true[0]), "converged": int(info.converged[0]),
           "pcg_ms": float(np.mean(pcg)), "gpu_launches_per_step": (api.launches() - L0) // steps,
           "roofline": {"bound": "hbm", "achieved": byts / pcg_s / 1e9, "peak": peaks()["hbm_gbs"],
                        "unit": "GB/s", "frac": byts / pcg_s / 1e9 / peaks()["hbm_gbs"], "traffic": None,
                        "kernel": "k_pcg_dense",
                        "note": "A (4.2 MB) and the operator stay in L2: the launch is bound by its "
                                "grid barriers, not by HBM"}}
    if cpu:
        import oracle
        oracle.build()
        c0 = time.perf_counter()
        S = oracle.Solve(mat, b[0], seed=1002, tol=1e-10)
        t = time.perf_counter() - c0
        out["cpu_baseline"] = {"value": 1.0 / t, "unit": "solves/s", "cores": 1, "kind": "oracle",
                               "sample": f"one complete oracle solve ({S.info['iters']} iterations)"}
        out["oracle_iters"] = int(S.info["iters"])
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_1806_02968_gb300 as pkg
    if rank == 0:
        pkg.build()
    if world > 1:
        dist.barrier()
    from paper_1806_02968_gb300 import api

    seed_base, seed_sample = replica_seeds(rank)
    mat, xs, b = make_problem(args, seed_base)
    m, n = mat["A"].shape
    A64 = torch.from_numpy(mat["A"]).cuda()
    bd = torch.from_numpy(b).cuda()
    M64 = api.Matrix(A64)
    if args.mode == "f64":
        es, es_res, es_op, pdt, dtype = 8, 8, 8, 0, "f64"
    elif args.mode == "f32":
        es, es_res, es_op, pdt, dtype = 4, 8, 4, 1, "f32+f64"
    else:
        es, es_res, es_op, pdt, dtype = 8, 8, 8, 0, "f32x2+f64"

    def solve_matrix(Asrc, Msrc):
        """The matrix the PCG iteration reads, derived from the FP64 input in-step."""
        if args.mode == "f64":
            return Msrc, None
        if args.mode == "f32":
            A32 = Asrc.float()
            return api.Matrix(A32, vals_f64=Asrc), A32
        pairs = api.lsq_split_f64(Asrc)
        return api.Matrix(pairs, f32x2=True, vals_f64=Asrc), pairs
    o = api.opts(seed=seed_sample, tol=args.tol, maxit=args.maxit, precond_dtype=pdt, sweeps=args.sweeps,
                 inner_tol=args.inner_tol, max_outer=50)
    stream = torch.cuda.current_stream()

    def step():
        idx, p, d = api.lsq_sample_rows(M64, o)
        P = api.lsq_build_precond(M64, idx, p, d, o)
        Mx, keep = solve_matrix(A64, M64)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = api.lsq_pcg_solve(Mx, P, bd, o)
        e1.record(stream)
        return x, info, (e0, e1)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    L0 = api.launches()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    pcg_ms, infos = [], []
    for _ in range(args.steps):
        x, info, (e0, e1) = step()
        infos.append(info)
        e1.synchronize()
        pcg_ms.append(e0.elapsed_time(e1))
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = api.launches() - L0
    ck = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    ms = max_over_ranks(ms, world, "cuda")
    ms_per_step = ms / args.steps
    value = whole_job_rate(world, args.steps, ms)

    info = infos[-1]
    byts, flops = pcg_algorithmic(args, m, n, info, es, es_res, es_op)
    pcg_s = float(np.mean(pcg_ms)) / 1e3
    pk = peaks()
    if args.mode == "f64":
        # FP64 FMA throughput bounds the fused pass on GB300 (2 FMAs per element of A per
        # iteration); the nominal FP64 rate 1.25 TFLOP/s is the denominator
        roof = {"bound": "alu", "achieved": flops / pcg_s / 1e12, "peak": 1.25, "unit": "TFLOP/s",
                "frac": flops / pcg_s / 1e12 / 1.25, "traffic": None,
                "hbm_gbs": byts / pcg_s / 1e9, "hbm_frac_of_measured": byts / pcg_s / 1e9 / pk["hbm_gbs"]}
    else:
        ratio = TRAFFIC_RATIO.get(args.mode)
        roof = {"bound": "hbm", "achieved": byts / pcg_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": byts / pcg_s / 1e9 / pk["hbm_gbs"],
                "traffic": byts * ratio if ratio else None}
        if ratio:
            roof["traffic_note"] = ("DRAM bytes per launch = algorithmic bytes x %.4f, the ratio "
                                    "measured by ncu on the 131072-row case of the same kernel" % ratio)
    roof["kernel"] = "k_pcg_dense"
    roof["peak_source"] = "MEASURED_PEAKS.json hbm_gbs (measured)" if args.mode != "f64" else \
        "nominal FP64 rate (152 SMs x 2 FMA/clk x 2.07 GHz); measured FMA probe 1.19 TFLOP/s"

    e2e = None
    if not args.no_e2e and rank == 0:
        hA = torch.empty_like(A64, device="cpu").pin_memory()
        hA.copy_(A64.cpu())
        hb = torch.from_numpy(b).pin_memory()
        hx = torch.empty(n, dtype=torch.float64).pin_memory()
        # every step: pinned host A and b to the device, the whole solve through the C ABI,
        # x back to pinned host memory; the mean over up to 3 steps (each is a full solve)
        e2e_steps = max(1, min(args.steps, 3))
        times = []
        for _ in range(e2e_steps):
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            dA = hA.to("cuda", non_blocking=True)
            db = hb.to("cuda", non_blocking=True)
            Mh64 = api.Matrix(dA)
            idx, p, d = api.lsq_sample_rows(Mh64, o)
            P = api.lsq_build_precond(Mh64, idx, p, d, o)
            Mh, keep = solve_matrix(dA, Mh64)
            xe, _ = api.lsq_pcg_solve(Mh, P, db, o)
            hx.copy_(xe, non_blocking=True)
            s1.record(stream)
            torch.cuda.synchronize()
            times.append(s0.elapsed_time(s1))
            del dA, db, Mh64, Mh, keep, P, xe
        e2e_ms = float(np.mean(times))
        e2e = {"value": 1e3 / e2e_ms, "unit": "solves/s", "h2d_bytes_per_step": int(hA.numel() * 8 + hb.numel() * 8),
               "d2h_bytes_per_step": int(n * 8), "steps": e2e_steps, "ms_per_step": e2e_ms}

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        t_solve, t_setup, t_iter = cpu_oracle_sample(mat, b, seed_sample, int(info.iters[0]), args.cpu_iters)
        cpu = {"value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle setup (sampling, A_s^T A_s, SGS) on the full matrix "
                         f"({t_setup:.2f} s) + {args.cpu_iters} PCG iterations ({t_iter:.3f} s each), "
                         f"extrapolated to the GPU's {int(info.iters[0])} iterations"}

    configs = None
    if rank == 0 and not args.no_configs and args.workload == "udv":
        configs = {}
        # the plain FP64 GPU solve of the same problem with the same samples: the comparison
        # point of the precision form (speed and error of every result against FP64)
        o64 = api.opts(seed=seed_sample, tol=args.tol, maxit=args.maxit, precond_dtype=0, sweeps=args.sweeps,
                       max_outer=50)
        idx, p, d = api.lsq_sample_rows(M64, o64)
        P64 = api.lsq_build_precond(M64, idx, p, d, o64)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        x64, info64 = api.lsq_pcg_solve(M64, P64, bd, o64)
        f1.record(stream)
        torch.cuda.synchronize()
        f64_ms = f0.elapsed_time(f1)
        err = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))
        fit = float(torch.linalg.norm(A64 @ (x - x64)) / torch.linalg.norm(A64 @ x64))
        it64 = int(info64.iters[0])
        b64 = it64 * (m * n * 8 + n * n * 8)
        configs[f"udv_dense_{m}x{n}_kappa{args.kappa:g}_f64"] = {
            "value": 1e3 / f64_ms, "unit": "solves/s (PCG only)", "pcg_ms": f64_ms, "dtype": "f64",
            "iters": it64, "relres_true": float(info64.relres_true[0]), "converged": int(info64.converged[0]),
            "roofline": {"bound": "alu", "achieved": it64 * (4.0 * m * n + 2.0 * n * n) / (f64_ms / 1e3) / 1e12,
                         "peak": 1.25, "unit": "TFLOP/s",
                         "frac": it64 * (4.0 * m * n + 2.0 * n * n) / (f64_ms / 1e3) / 1e12 / 1.25,
                         "traffic": None, "kernel": "k_pcg_dense (FP64 values)",
                         "hbm_gbs": b64 / (f64_ms / 1e3) / 1e9},
            "speedup_of_headline_form": f64_ms / float(np.mean(pcg_ms))}
        err_vs_f64 = {"rel_x": err, "rel_Ax": fit, "f64_iters": it64,
                      "note": "||x - x_f64|| / ||x_f64|| and ||A (x - x_f64)|| / ||A x_f64|| against the "
                              "FP64 GPU solve with the same samples; both meet the relative normal-equation "
                              "residual 1e-10, which at kappa(A) = 1e6 leaves the components along the "
                              "smallest singular directions free up to kappa^2 tol"}
        gc.collect()
        torch.cuda.empty_cache()
        configs["gaussian_dense_4096x128"] = gauss_config(cpu=not args.no_cpu_baseline)
        for w in ("sparse", "graph", "adjoint"):
            c = sparse_config(w, cpu=not args.no_cpu_baseline)
            configs[c["config"]["workload"]] = c
            gc.collect()
            torch.cuda.empty_cache()
        configs["uneven_dense_batch_64x16rhs"] = batch_config(cpu=not args.no_cpu_baseline)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
                "data": "synthetic",
                "config": {"workload": workload_name(args, m, n), "m": m, "n": n,
                           "kappa": args.kappa, "tol": args.tol, "sweeps": args.sweeps, "s": int(info.s),
                           "mode": args.mode, "l2": "inputs larger than L2 (A is %.2f GB)" % (m * n * es / 1e9),
                           "parallelism": f"replicas{world}"},
                "clocks": ck, "gpu_launches": int(launches),
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
                "solve": {"iters": int(info.iters[0]), "outer": int(info.outer[0]),
                          "relres_true": float(info.relres_true[0]),
                          "relres_raw": float(info.relres_raw[0]),
                          "converged": int(info.converged[0]), "pcg_ms": float(np.mean(pcg_ms)),
                          "us_per_iter": 1e3 * float(np.mean(pcg_ms)) / max(int(info.iters[0]), 1)}}
        if configs is not None:
            line["err_vs_f64"] = err_vs_f64
            line["configs"] = configs
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


SPARSE_CFGS = {
    # name: (generator, right-hand sides, noise, value type)
    "sparse": ("sparse_random_4000000x40000_8nnz", 1, 1e-3, "f32"),
    "graph": ("graph_incidence_262144nodes_32rhs", 32, 1e-4, "f64"),
    "adjoint": ("sparse_random_1000000x10000_16rhs_adjoint", 16, 1e-3, "f32"),
}


def sparse_matrix(which):
    import workloads as W
    if which == "sparse":
        return W.sparse_random(4_000_000, 40_000, 8, 3)
    if which == "graph":
        return W.graph_incidence(262144, 8 * 262144, 4)
    return W.sparse_random(1_000_000, 10_000, 8, 5)


def csr_bytes_per_iter(mat, nnz_m, es, k):
    """Algorithmic bytes of one CSR PCG iteration: A once (values, column indices, row
    pointers), M = A_s^T A_s once over the two sweeps (values and indices), and about ten
    n x k FP64 vector passes."""
    m, n = int(mat["m"]), int(mat["n"])
    nnz_a = int(mat["row_ptr"][-1])
    return nnz_a * (es + 4) + 8 * (m + 1) + nnz_m * (es + 4) + 8 * (n + 1) + 10 * 8 * n * k


def oracle_csr_sample(mat, b, seed, iters_gpu, k, cpu_iters=3):
    """Oracle (FP64, one thread) on one column of the same input: full setup (S1-S6) plus
    cpu_iters PCG iterations, extrapolated to the GPU's iterations and k columns."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    smp = oracle.Sample(mat, seed)
    Mo = oracle.SampledM(smp)
    t1 = time.perf_counter()
    oracle.pcg(smp.mat, smp.d, Mo, b=b, tol=1e-300, maxit=cpu_iters, max_outer=1)
    t2 = time.perf_counter()
    per_iter = (t2 - t1) / cpu_iters
    t = (t1 - t0) + per_iter * max(iters_gpu, 1) * k
    return {"value": k / t, "unit": "solves/s (right-hand sides)", "cores": 1, "kind": "oracle",
            "sample": f"oracle setup (sampling, A_s^T A_s) on the full matrix ({t1 - t0:.1f} s) + "
                      f"{cpu_iters} PCG iterations of one column ({per_iter:.3f} s each), extrapolated "
                      f"to the GPU's {iters_gpu} iterations x {k} columns"}


def sparse_config(which, tol=1e-10, maxit=1000000, sweeps=1, inner_tol=0.0, steps=3, warmup=1,
                  cpu=True, mat=None, device_loop=0):
    """One CSR configuration: sparse random 4e6 x 4e4 (FP32 values, FP64 refinement), weighted
    graph incidence with 32 right-hand sides (FP64), or sparse 1e6 x 1e4 with 16 right-hand
    sides through the solve and the adjoint (FP32 values, FP64 refinement).  A step is
    sampling, the preconditioner and the solve (and the adjoint), timed with synchronising
    host clocks around each phase."""
    import torch
    import workloads as W
    from paper_1806_02968_gb300 import api
    name, k, noise, dt = SPARSE_CFGS[which]
    mat = mat if mat is not None else sparse_matrix(which)
    xs, b = W.rhs_for(mat, k, noise, 1234)
    rp = torch.from_numpy(mat["row_ptr"]).cuda()
    ci = torch.from_numpy(mat["col_idx"]).cuda()
    v64 = torch.from_numpy(mat["vals"]).cuda()
    vals = v64.float() if dt == "f32" else v64
    Mx = api.Matrix(row_ptr=rp, col_idx=ci, vals=vals, n=mat["n"], vals_f64=v64 if dt == "f32" else None)
    o = api.opts(seed=1003, tol=tol, maxit=maxit, max_outer=50, inner_tol=inner_tol, sweeps=sweeps,
                 precond_dtype=1 if dt == "f32" else 0, device_loop=device_loop)
    B = torch.from_numpy(b).cuda()
    # the graph configuration is defined as one persistent launch inside a captured CUDA graph
    captured = which == "graph"
    if captured:
        o.device_loop = 1
        cap_stream = torch.cuda.Stream()
        cap_stream.wait_stream(torch.cuda.current_stream())
        # one direct call first: its per-column results are the ones reported (a captured call
        # reports none), and it sets up the launch outside the capture
        idx0, p0, d0 = api.lsq_sample_rows(Mx, o)
        P0 = api.lsq_build_precond(Mx, idx0, p0, d0, o)
        _, info = api.lsq_pcg_solve(Mx, P0, B, o)
        del P0
    runs = []
    L0 = api.launches()
    for rep in range(warmup + steps):
        if rep == warmup:
            L0 = api.launches()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idx, p, d = api.lsq_sample_rows(Mx, o)
        torch.cuda.synchronize(); t1 = time.perf_counter()
        P = api.lsq_build_precond(Mx, idx, p, d, o)
        torch.cuda.synchronize(); t2 = time.perf_counter()
        if captured:
            # the solve as one persistent launch captured in a CUDA graph, then replayed
            X = torch.empty(k, mat["n"], dtype=torch.float64, device="cuda")
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(cap_stream):
                with torch.cuda.graph(g, stream=cap_stream):
                    api.lsq_pcg_solve(Mx, P, B, o, X=X, stream=cap_stream)
            g.replay()
            torch.cuda.synchronize(); t3 = time.perf_counter()
        else:
            X, info = api.lsq_pcg_solve(Mx, P, B, o)
            torch.cuda.synchronize(); t3 = time.perf_counter()
        r = {"sample_s": t1 - t0, "build_s": t2 - t1, "solve_s": t3 - t2}
        if which == "adjoint":
            G = 2 * (X - torch.from_numpy(xs).cuda())
            gb, gv, lam, ainfo = api.lsq_pcg_adjoint(Mx, P, X, B, G, o)
            torch.cuda.synchronize()
            r["adjoint_s"] = time.perf_counter() - t3
            r["adjoint_iters_max"] = int(np.max(ainfo.iters))
        if rep >= warmup:
            runs.append(r)
    launches = (api.launches() - L0) // max(steps, 1)
    res = {key: float(np.mean([r[key] for r in runs])) for key in runs[0]}
    tot = res["sample_s"] + res["build_s"] + res["solve_s"] + res.get("adjoint_s", 0.0)
    it = int(np.max(info.iters))
    es = 4 if dt == "f32" else 8
    per_iter = csr_bytes_per_iter(mat, int(info.nnz_M), es, k)
    achieved = it * per_iter / res["solve_s"] / 1e9
    out = {"value": k / tot, "unit": "solves/s (right-hand sides)", "ms_per_step": tot * 1e3,
           "steps": steps, "warmup": warmup, "dtype": dt + ("+f64" if dt == "f32" else ""),
           "config": {"workload": name, "m": int(mat["m"]), "n": int(mat["n"]), "k": k, "tol": tol,
                      "sweeps": sweeps, "device_loop": int(o.device_loop),
                      "solve_form": "captured CUDA graph, one persistent launch" if captured else
                                    ("one persistent launch" if o.device_loop else "stream-ordered kernels"),
                      "nnz_A": int(mat["row_ptr"][-1]), "nnz_M": int(info.nnz_M),
                      "levels": int(info.levels), "s": int(info.s)},
           "iters_max": it, "iters": info.iters.tolist() if k <= 4 else None,
           "converged": int(np.sum(info.converged)), "relres_true_max": float(np.max(info.relres_true)),
           "gpu_launches_per_step": int(launches),
           "phases": res,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks()["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved / peaks()["hbm_gbs"], "traffic": None,
                        "kernel": "whole CSR iteration (row and column passes, sweeps, vector kernels)",
                        "bytes_per_iter": per_iter,
                        "note": "algorithmic bytes per iteration (A once, M once, ~10 n x k vector "
                                "passes) x iterations / solve time"}}
    if sweeps > 0:
        out["sweep"] = sweep_latency_bound(api, P, mat["n"], sweeps, int(info.levels))
    if cpu:
        out["cpu_baseline"] = oracle_csr_sample(mat, b[0], 1003, it, k)
    return out


def sweep_latency_bound(api, P, n, sweeps, levels, reps=3):
    """The one-column Gauss-Seidel sweep (Alg. 3) against its latency bound: a sweep is a chain
    of `levels` levels, each needing at least one hand-off of a value between SMs (half the
    measured round trip) and one dependent load of it (an L2 load).  The sweep time is the
    preconditioner application (t forward + t backward sweeps) over 2t, CUDA events."""
    import torch
    lat = api.measure_latency()
    R = torch.randn(n, dtype=torch.float64, device="cuda")
    P.apply(R)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        P.apply(R)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps / (2 * sweeps)
    per_level_ns = 0.5 * lat["sm_round_trip_ns"] + lat["l2_load_ns"]
    bound = levels * per_level_ns / 1e6
    return {"ms_per_sweep": ms, "levels": levels, "us_per_level": 1e3 * ms / max(levels, 1),
            "latency_ns": lat, "bound": "latency", "bound_ms_per_sweep": bound,
            "frac": bound / ms if ms > 0 else None,
            "note": "bound = levels x (half an SM-to-SM round trip + one dependent L2 load), measured "
                    "on this device by lsq_measure_latency; sweep = one-column preconditioner "
                    "application / 2t"}


def run_sparse_workload(args):
    import torch
    import paper_1806_02968_gb300 as pkg
    from paper_1806_02968_gb300 import api
    pkg.build()
    torch.cuda.set_device(0)
    api.set_sweep_form(args.sweep_form)
    out = sparse_config(args.workload, args.tol, args.maxit, args.sweeps, args.inner_tol,
                        args.steps, args.warmup, cpu=not args.no_cpu_baseline, device_loop=args.device_loop)
    line = {"metric": METRIC, "n_gpus": 1, "higher_is_better": True, "data": "synthetic", **out}
    print(json.dumps(line), flush=True)


# FP32 FMA peak of the batch kernel's arithmetic: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def batch_config(tol=1e-10, maxit=1000000, steps=5, warmup=3, cpu=True):
    """64 uneven dense Gaussian problems (m log-uniform in [1024, 16384], n in [32, 256]),
    16 right-hand sides each, FP32 values: all PCG solves in one launch (lsq_batch_solve,
    replayed from a captured CUDA graph), against the same problems solved one at a time
    with FP64 values (lsq_pcg_solve)."""
    import torch
    import workloads as W
    from paper_1806_02968_gb300 import api

    class _A:
        pass
    args = _A()
    args.tol, args.maxit, args.steps, args.warmup = tol, maxit, steps, warmup
    count, k = 64, 16
    mats = W.uneven_dense_batch(count, (1024, 16384), (32, 256), 5)
    o = api.opts(tol=args.tol, maxit=min(args.maxit, 100000), max_outer=30, inner_tol=1e-4)
    probs, keep = [], []
    t0 = time.perf_counter()
    for i, mt in enumerate(mats):
        A64 = np.asarray(mt["A"])
        m, n = A64.shape
        ld = (n + 3) // 4 * 4
        T = torch.zeros(m, ld, dtype=torch.float32, device="cuda")
        T[:, :n] = torch.from_numpy(A64).float().cuda()
        seen = {"kind": "dense", "A": T[:, :n].double().cpu().numpy()}
        xs, b = W.rhs_for(seen, k, 1e-3, 100 + i)
        keep.append((T, seen, torch.from_numpy(b).cuda()))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for i, (T, seen, B) in enumerate(keep):
        n = seen["A"].shape[1]
        Mx = api.Matrix(T[:, :n])
        po = api.opts(seed=200 + i, precond_dtype=1)
        idx, p, d = api.lsq_sample_rows(Mx, po)
        P = api.lsq_build_precond(Mx, idx, p, d, po)
        probs.append((T, n, P, B))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    bt = api.Batch(probs, o)
    cluster = bt.autotune()
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    Lc0 = api.launches()
    with torch.cuda.stream(stream):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            bt.solve(stream=stream)
    torch.cuda.synchronize()
    kernels_per_replay = api.launches() - Lc0   # kernels in the captured graph
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1) / args.steps
    infos = bt.info()
    iters = np.array([inf.iters for inf in infos])
    outers = np.array([inf.outer for inf in infos])
    conv = np.array([inf.converged for inf in infos])
    tru = np.array([inf.relres_true for inf in infos])
    # algorithmic work of one launch: per problem, one pass over A (FP32) per inner iteration
    # of its slowest column and one FP64 residual pass per (re)start plus the final check
    byts, flops = 0.0, 0.0
    for (T, n, P, B), it, ou in zip(probs, iters, outers):
        m = T.shape[0]
        passes = int(it.max()) + int(ou.max()) + 1
        byts += passes * m * T.shape[1] * 4.0
        flops += int(it.max()) * 4.0 * m * n * k
    # the same problems, one at a time, FP64 values (the plain GPU solve), solves only
    singles = []
    for i, (T, seen, B) in enumerate(keep):
        m, n = seen["A"].shape
        A64 = torch.zeros(m, n + (n & 1), dtype=torch.float64, device="cuda")   # 16-byte rows
        A64[:, :n] = torch.from_numpy(seen["A"]).cuda()
        M64 = api.Matrix(A64[:, :n])
        po = api.opts(seed=200 + i)
        idx, p, d = api.lsq_sample_rows(M64, po)
        singles.append((A64, M64, api.lsq_build_precond(M64, idx, p, d, po), B))
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f64_iters = []
    f0.record()
    for A64, M64, P64, B in singles:
        X64, inf64 = api.lsq_pcg_solve(M64, P64, B, api.opts(tol=args.tol))
        f64_iters.append(int(inf64.iters.max()))
    f1.record()
    torch.cuda.synchronize()
    f64_ms = f0.elapsed_time(f1)
    out = {"value": count * k / (solve_ms / 1e3), "unit": "solves/s (right-hand sides)",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": solve_ms, "dtype": "f32+f64",
            "config": {"workload": "uneven_dense_batch_64x16rhs", "count": count, "k": k,
                       "m_range": [1024, 16384], "n_range": [32, 256], "tol": args.tol,
                       "A_bytes": int(sum(T.numel() * 4 for T, _, _, _ in probs)), "cluster": cluster,
                       "l2": "A (about the L2 size) stays resident across replays"},
            "gpu_launches_per_step": kernels_per_replay,
            "roofline": {"bound": "alu", "achieved": flops / (solve_ms / 1e3) / 1e12,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops / (solve_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS, "traffic": None,
                         "kernel": "k_pcg_batch", "hbm_gbs": byts / (solve_ms / 1e3) / 1e9,
                         "peak_source": "nominal FP32 FMA rate (152 SMs x 128 lanes x 2 x 2.07 GHz)"},
            "phases": {"gen_s": t1 - t0, "setup_s": t2 - t1, "plan_autotune_s": t3 - t2,
                       "solve_ms": solve_ms, "iters_max": int(iters.max()), "iters_mean": float(iters.mean()),
                       "outer_max": int(outers.max()), "converged": int(conv.sum()),
                       "relres_true_max": float(tru.max()),
                       "f64_one_at_a_time_ms": f64_ms, "f64_iters_mean": float(np.mean(f64_iters)),
                       "speedup_vs_f64_single": f64_ms / solve_ms}}
    if cpu:
        # the oracle on 4 of the 64 problems, one right-hand side each, scaled to 64 x 16
        import oracle
        oracle.build()
        picks = [0, 21, 42, 63]
        t0 = time.perf_counter()
        for i in picks:
            T, seen, B = keep[i]
            S = oracle.Solve(seen, B[0].cpu().numpy(), seed=200 + i, tol=tol, max_outer=30)
        t_cpu = (time.perf_counter() - t0) * (count / len(picks)) * k
        out["cpu_baseline"] = {"value": count * k / t_cpu, "unit": "solves/s (right-hand sides)", "cores": 1,
                               "kind": "oracle",
                               "sample": f"oracle end to end (setup + FP64 PCG) on problems {picks}, one "
                                         f"right-hand side each, scaled to {count} problems x {k} columns"}
    return out


def run_batch_workload(args):
    import torch
    import paper_1806_02968_gb300 as pkg
    pkg.build()
    torch.cuda.set_device(0)
    out = batch_config(args.tol, args.maxit, args.steps, args.warmup, cpu=not args.no_cpu_baseline)
    print(json.dumps({"metric": METRIC, "n_gpus": 1, "higher_is_better": True, "data": "synthetic", **out}),
          flush=True)


def tc_grid(steps=3, warmup=1):
    """Sweeps t in {1, 2, 5} (and t = 0, CG on the normalised A) against the sample factor
    C in {2, 4, 8} (s = ceil(C n ln n)): iterations and time to 1e-10 of a whole solve
    (sampling, preconditioner, PCG) on a Gaussian 4096 x 128, a UDV 20000 x 256 with
    kappa(A) = 1e3 and a sparse random 100000 x 2000 (8 per row), FP64, one right-hand side
    b = A x* + 1e-3 N(0,1).  Each setting is timed over `steps` solves after `warmup`."""
    import torch
    import workloads as W
    from paper_1806_02968_gb300 import api
    mats = {"gaussian_dense_4096x128": W.gaussian_dense(4096, 128, 7),
            "udv_dense_20000x256_kappa1e3": W.udv_dense(20000, 256, 1e3, 7),
            "sparse_random_100000x2000_8nnz": W.sparse_random(100000, 2000, 8, 7)}
    out = {}
    for name, mat in mats.items():
        xs, b = W.rhs_for(mat, 1, 1e-3, 8)
        if mat["kind"] == "dense":
            A = torch.from_numpy(mat["A"]).cuda()
            Mx, keep = api.Matrix(A), [A]
        else:
            keep = [torch.from_numpy(mat[k]).cuda() for k in ("row_ptr", "col_idx", "vals")]
            Mx = api.Matrix(row_ptr=keep[0], col_idx=keep[1], vals=keep[2], n=mat["n"])
        B = torch.from_numpy(b[0]).cuda()
        rows = {}
        for t in (0, 1, 2, 5):
            for C in (2.0, 4.0, 8.0):
                if t == 0 and C != 4.0:
                    continue      # CG does not sample
                o = api.opts(seed=11, sweeps=t, sample_factor=C)
                times = []
                for rep in range(warmup + steps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    idx, p, d = api.lsq_sample_rows(Mx, o)
                    P = api.lsq_build_precond(Mx, idx, p, d, o)
                    x, info = api.lsq_pcg_solve(Mx, P, B, o)
                    torch.cuda.synchronize()
                    if rep >= warmup:
                        times.append(time.perf_counter() - t0)
                rows[f"t={t},C={C:g}"] = {"iters": int(info.iters[0]), "ms": 1e3 * float(np.mean(times)),
                                          "relres_true": float(info.relres_true[0]), "s": int(info.s)}
        out[name] = rows
    return out


def sampling_cmp(steps=3, warmup=1):
    """The method's row density (squared norms, Eq. R2P) against uniform sampling (the
    comparison of Sec. 3.1) and against CG on the normalised A, on matrices whose rows differ:
    400 heavy Gaussian rows among 20000 (the rest scaled by 1e-3), the sparse random
    4,000,000 x 40,000 configuration (per-row scales 10^U(-2, 2); FP32 values, FP64 restarts),
    and the semi-Gaussian [B 0; 0 I] of Sec. 5.2 (coherent, but its identity block is already
    its own normal matrix).  Iterations and time to 1e-10 of a whole solve."""
    import torch
    import workloads as W
    from paper_1806_02968_gb300 import api
    rng = np.random.default_rng(4)
    heavy = rng.standard_normal((20000, 100))
    heavy[400:] *= 1e-3
    mats = {"heavy_rows_dense_20000x100": ({"kind": "dense", "A": heavy}, "f64"),
            "sparse_random_4000000x40000_8nnz": (sparse_matrix("sparse"), "f32"),
            "semi_gaussian_dense_10000x200": (W.semi_gaussian_dense(10000, 200, 21), "f64")}
    out = {}
    for name, (mat, dt) in mats.items():
        xs, b = W.rhs_for(mat, 1, 1e-3, 6)
        if mat["kind"] == "dense":
            A = torch.from_numpy(mat["A"]).cuda()
            Mx, keep, pdt = api.Matrix(A), [A], 0
        else:
            keep = [torch.from_numpy(mat[k]).cuda() for k in ("row_ptr", "col_idx", "vals")]
            v = keep[2].float() if dt == "f32" else keep[2]
            keep.append(v)
            Mx = api.Matrix(row_ptr=keep[0], col_idx=keep[1], vals=v, n=mat["n"],
                            vals_f64=keep[2] if dt == "f32" else None)
            pdt = 1 if dt == "f32" else 0
        B = torch.from_numpy(b[0]).cuda()
        rows = {}
        for label, sampling, sweeps in (("norm2", 0, 1), ("uniform", 1, 1), ("cg", 0, 0)):
            o = api.opts(seed=5, sweeps=sweeps, sampling=sampling, precond_dtype=pdt, max_outer=50)
            times = []
            for rep in range(warmup + steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                idx, p, d = api.lsq_sample_rows(Mx, o)
                P = api.lsq_build_precond(Mx, idx, p, d, o)
                x, info = api.lsq_pcg_solve(Mx, P, B, o)
                torch.cuda.synchronize()
                if rep >= warmup:
                    times.append(time.perf_counter() - t0)
            rows[label] = {"iters": int(info.iters[0]), "ms": 1e3 * float(np.mean(times)),
                           "relres_true": float(info.relres_true[0]), "unsampled_columns": int(info.n_fixed_diag)}
        out[name] = rows
    return out


def run_sampling(args):
    import torch
    import paper_1806_02968_gb300 as pkg
    pkg.build()
    torch.cuda.set_device(0)
    print(json.dumps({"metric": METRIC, "unit": "ms per solve (sampling + preconditioner + PCG)",
                      "n_gpus": 1, "data": "synthetic", "tol": 1e-10,
                      "comparison": sampling_cmp(args.steps, args.warmup)}), flush=True)


# The paper's own tables (Sec. 5.1, 5.2, 5.4, 5.5): its sizes, t = 5 sweeps, tolerance 1e-7,
# s = ceil(4 n ln n), b ~ N(0, 1).  Printed values: iterations of CG on the normalised A and
# of PCG with the row-sampling preconditioner (RS; a mean over ten runs where the paper gives one).
PAPER_TABLES = {
    "gaussian": [((3000, 109), 10, 11), ((5000, 141), 9, 11), ((10000, 200), 9, 11),
                 ((20000, 282), 8, 11), ((40000, 400), 7, 10.9)],
    "semi_gaussian": [((1000, 62), 9, 11.7), ((3000, 108), 8, 11.7), ((5000, 140), 8, 11.9),
                      ((10000, 200), 7, 11.7), ((20000, 282), 7, 11.3)],
    # kappa(A^T A) as printed; D linear from 1 to sqrt(kappa)
    "udv_linear_90000x300": [(5936, 116, 23.1), (18853, 202, 38.8), (1.44e5, 294, 72),
                             (4.75e5, 369, 86.4), (1.07e6, 253, 90.2)],
    # vertices per glued graph (2 n - 5 vertices: 187 ... 856 in the paper's table)
    "graph_laplacian_chung_lu": [(96, 40, 16.7), (180, 67, 21.9), (270, 60, 21), (357, 93, 26.8), (430, 112, 30.2)],
}


def paper_tables(steps=1, warmup=1, seeds=5):
    """Every family of the paper's iteration tables on the GPU, at the printed sizes and
    settings: CG iterations, RS iterations for `seeds` sampling seeds, and the time of a whole
    solve (sampling, preconditioner, PCG) for each, beside the printed iteration counts."""
    import torch
    import workloads as W
    from paper_1806_02968_gb300 import api
    out = {}
    for fam, rows in PAPER_TABLES.items():
        res = []
        for key, cg_paper, rs_paper in rows:
            if fam == "gaussian":
                mat = W.gaussian_dense(key[0], key[1], 1)
            elif fam == "semi_gaussian":
                mat = W.semi_gaussian_dense(key[0], key[1], 1)
            elif fam.startswith("udv"):
                mat = W.udv_dense(90000, 300, float(np.sqrt(key)), 1, spacing="linear")
            else:
                mat = W.chung_lu_incidence(key, 5)
            if mat["kind"] == "dense":
                m, n = mat["A"].shape
                # rows start on 16-byte boundaries (the row copies' alignment): pad odd n
                A = torch.zeros(m, n + (n & 1), dtype=torch.float64, device="cuda")
                A[:, :n] = torch.from_numpy(mat["A"]).cuda()
                Mx, keep = api.Matrix(A[:, :n]), [A]
            else:
                m, n = mat["m"], mat["n"]
                keep = [torch.from_numpy(mat[k]).cuda() for k in ("row_ptr", "col_idx", "vals")]
                Mx = api.Matrix(row_ptr=keep[0], col_idx=keep[1], vals=keep[2], n=n)
            B = torch.from_numpy(np.random.default_rng(1).standard_normal(m)).cuda()
            row = {"m": m, "n": n, "iters_cg_paper": cg_paper, "iters_rs_paper": rs_paper}
            for label, sweeps, seed_list in (("cg", 0, [1]), ("rs", 5, list(range(1, seeds + 1)))):
                its, ms, rr, ok = [], [], [], []
                for seed in seed_list:
                    o = api.opts(seed=seed, sweeps=sweeps, tol=1e-7, max_outer=20)
                    times = []
                    for rep in range(warmup + steps):
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        idx, p, d = api.lsq_sample_rows(Mx, o)
                        P = api.lsq_build_precond(Mx, idx, p, d, o)
                        x, info = api.lsq_pcg_solve(Mx, P, B, o)
                        torch.cuda.synchronize()
                        if rep >= warmup:
                            times.append(time.perf_counter() - t0)
                    its.append(int(info.iters[0]))
                    ms.append(1e3 * float(np.mean(times)))
                    rr.append(float(info.relres_true[0]))
                    ok.append(int(info.converged[0]))
                    row["s"] = int(info.s)
                row[f"iters_{label}"] = its if label == "rs" else its[0]
                row[f"ms_{label}"] = float(np.mean(ms))
                row[f"relres_true_{label}_max"] = max(rr)
                row[f"converged_{label}"] = int(min(ok))
            res.append(row)
        out[fam] = res
    return out


def run_paper(args):
    import torch
    import paper_1806_02968_gb300 as pkg
    pkg.build()
    torch.cuda.set_device(0)
    print(json.dumps({"metric": METRIC, "unit": "iterations; ms per solve (sampling + preconditioner + PCG)",
                      "n_gpus": 1, "data": "synthetic", "dtype": "f64", "tol": 1e-7, "sweeps": 5,
                      "tables": paper_tables(args.steps, args.warmup)}), flush=True)


def run_tc(args):
    import torch
    import paper_1806_02968_gb300 as pkg
    pkg.build()
    torch.cuda.set_device(0)
    print(json.dumps({"metric": METRIC, "unit": "ms per solve (sampling + preconditioner + PCG)",
                      "n_gpus": 1, "data": "synthetic", "dtype": "f64", "tol": 1e-10,
                      "grid": tc_grid(args.steps, args.warmup)}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch_workload(args)
    elif args.workload == "tc":
        run_tc(args)
    elif args.workload == "sampling":
        run_sampling(args)
    elif args.workload == "paper":
        run_paper(args)
    elif args.workload not in ("udv", "gauss"):
        run_sparse_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
