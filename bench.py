#!/usr/bin/env python
"""Benchmark: TV-superiorized CG reconstructions per second on GB300.

One step = one complete solve of the hot path to the stopping threshold: the
projector A and backprojector A^T (2 + 2 passes per S-CG loop body), the TV
subgradient and TV trial passes of the perturbation step, the CG scalars and
vector updates, and the eps test -- on one batch (one problem) of seeded
synthetic input already resident in HBM.

Default workload: 512x512 ellipse phantom (20 ellipses), 720 angles x 725
bins, noise sigma = 0.5 % of max(Ax), eps = 1.05 * L sigma^2 / 2, FP32
storage/arithmetic with FP64 reductions and scalars, variant S-CG.  The
problem state (~20 MB) fits in L2, so the L2 is flushed (a 512 MiB write)
before every timed step, outside the step's event pair.

The sinogram of both arms is built with the FP64 oracle's projector (the
same y, eps and config for ``--impl ours`` and ``--impl reference``).

Beside the headline the line carries a ``batch`` block (the 256-problem
uneven batch recipe through scg_solve_batch in binary16 storage, against the
same problems solved one by one on the plain FP32 single-solve path) and a
``serving`` block (a Poisson stream of few-view requests through the
continuous-batching server in binary16: achieved rate, p50/p99 latency, the
saturated rate against FP32 solo solves), each with its own clocks.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead: whole solves of the same problem, as many as fit a bounded
CPU budget.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1709_04912_gb300 import inputs  # noqa: E402

METRIC = "S-CG recon/s at fixed eps"
UNIT = "recon/s"
# FP32 lane operations per nonzero ray-pixel weight of the projector pair's
# roofline: 10, the cost of evaluating one chord weight from its definition and
# accumulating it (signed distance of the pixel centre from the ray 2, |d| 1, the
# two clips of the trapezoid 2, the scale 1/(m n) 1, the select of the
# axis-aligned case 1, the multiply-add into the ray sum 1, the index 2).  The
# kernels need fewer (the walk makes the distance an increment and the clips one
# saturate); the line also reports the fraction at the minimum of 7 (position 2,
# distance 1, weight 3, accumulation 1).
OPS_PER_NNZ = 10
OPS_PER_NNZ_MIN = 7
WORKLOADS = {w.name: w for w in (inputs.SINGLE_512, inputs.SMALL_FP64, inputs.MIXED_1024,
                                  inputs.PAPER_512)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="S-CG")
    ap.add_argument("--workload", default=inputs.SINGLE_512.name, choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--gamma0-rel", type=float, default=0.05)
    ap.add_argument("--lam", type=float, default=30.0, help="FISTA's TV weight lambda (--variant FISTA)")
    ap.add_argument("--prox-iters", type=int, default=10,
                    help="FGP steps per prox (--variant FISTA, --perturb prox)")
    ap.add_argument("--perturb-steps", type=int, default=1,
                    help="perturbations per step of the S-variants (scg_params.perturb_steps)")
    ap.add_argument("--perturb", default="gamma", choices=["gamma", "prox"],
                    help="superiorization rule of the S-variants: the gamma rule with its TV test, or the "
                         "proximal perturbation prox_{lambda TV}(x_k)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="leave the batch block out of the line")
    ap.add_argument("--no-serving", action="store_true", help="leave the serving block out of the line")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="CPU seconds the reference arm spends on timed oracle solves")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serving"],
                    help="single: the headline solve; batch: uneven batch through scg_solve_batch "
                         "vs the same solves one by one; serving: Poisson request stream through "
                         "the continuous-batching server")
    ap.add_argument("--batch", type=int, default=256, help="problems in --mode batch")
    ap.add_argument("--rate", type=float, default=None,
                    help="requests/s of the Poisson stream (--mode serving 50, serving block 200)")
    ap.add_argument("--duration", type=float, default=None,
                    help="measured seconds of the Poisson stream (--mode serving 20, serving block 8)")
    ap.add_argument("--serve-warmup", type=float, default=None,
                    help="warm-up seconds of the Poisson stream (--mode serving 5, serving block 2)")
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--pool-gb", type=float, default=16.0)
    ap.add_argument("--dtype", default=None, choices=["f32", "f16", "bf16", "f64"],
                    help="storage precision: single and batch modes default to f32, serving to f16")
    ap.add_argument("--host-loop", action="store_true",
                    help="run the while loop as host-polled per-body graphs (same kernels); "
                         "lets a profiler list every kernel launch")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def barrier(world):
    """Every rank reaches this point before any goes on (no-op for one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(t_local: float, world: int, device=None) -> float:
    """The slowest rank's time: the whole job's time for replicas that each
    process their own problems."""
    if world == 1:
        return float(t_local)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank: int, world: int, t_max: float) -> float:
    """Units all ranks processed per second of the slowest rank's time."""
    return units_per_rank * world / t_max


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def nnz_of(work) -> int:
    """Exact number of nonzero ray-pixel weights of A (one count per angle)."""
    n, na, nb = work.n, work.n_angles, work.n_bins
    idx = np.arange(n) - 0.5 * (n - 1)
    yc, xc = np.meshgrid(idx, idx, indexing="ij")
    total = 0
    for a in range(na):
        if a == 0:
            c, s = 1.0, 0.0
        elif 2 * a == na:
            c, s = 0.0, 1.0
        else:
            c, s = math.cos(math.pi * a / na), math.sin(math.pi * a / na)
        m, mn = max(abs(c), abs(s)), min(abs(c), abs(s))
        hs = 0.5 * (m + mn)
        cb = (xc * c + yc * s + 0.5 * (nb - 1)).ravel()
        if mn == 0.0:       # closed window of half-width 1/2 (edge rays count for both pixels)
            lo = np.ceil(cb - 0.5)
            hi = np.floor(cb + 0.5)
        else:               # open window (cb - hs, cb + hs)
            lo = np.floor(cb - hs) + 1
            hi = np.ceil(cb + hs) - 1
        lo = np.maximum(lo, 0)
        hi = np.minimum(hi, nb - 1)
        total += int(np.sum(np.maximum(hi - lo + 1, 0)))
    return total


# ---------------------------------------------------------------------------
def time_oracle_solves(prob, work, variant, gamma0_rel, budget_s, max_solves, lam=0.0, prox_iters=10,
                       perturb="gamma", perturb_steps=1, warmup=0):
    """Whole oracle solves of ``prob`` (FP64, on the host cores): ``warmup``
    untimed ones, then solves timed one by one until ``budget_s`` seconds (the
    warm-up included; at least one timed solve) or ``max_solves`` solves.
    Returns the times, the iteration count and the thread count.  FISTA's c^2 comes from the oracle's own power iteration (100
    steps, the library's count), outside the timed solves."""
    import oracle
    kw = dict(variant=variant, gamma0_rel=gamma0_rel, eps=prob.eps, max_iter=work.max_iter)
    if variant in ("CG", "PCG"):
        kw["perturb"] = "none"
    elif perturb == "prox":
        kw.update(perturb="prox", prox_iters=prox_iters)
    if variant not in ("CG", "PCG", "FISTA") and perturb_steps > 1:
        kw["perturb_steps"] = perturb_steps
    if variant == "FISTA":
        c2 = oracle.norm_A(work.n, work.n_angles, work.n_bins, 100) ** 2

        def one():
            return oracle.fista(prob.y, work.n, prob.eps, lam, c2, prox_iters=prox_iters, max_iter=300)
    else:
        oracle.solve(prob.y, work.n, **dict(kw, max_iter=0))  # loads the library

        def one():
            return oracle.solve(prob.y, work.n, **kw)
    t_all = time.perf_counter()
    for _ in range(max(0, warmup)):
        one()
    times, iters = [], 0
    while len(times) < max(1, max_solves):
        t0 = time.perf_counter()
        _, res, _ = one()
        times.append(time.perf_counter() - t0)
        iters = res["iters"]
        if time.perf_counter() - t_all >= budget_s:
            break
    return times, iters, oracle.num_threads()


def run_reference(args, work, rank, world):
    """The FP64 CPU oracle: whole solves of the same problem as ours."""
    if rank != 0:
        return 0
    import oracle
    variant = args.variant
    prob = inputs.make_problem(work, args.seed, oracle.project)
    times, iters, cores = time_oracle_solves(prob, work, variant, args.gamma0_rel, args.ref_budget, args.steps,
                                             args.lam, args.prox_iters, args.perturb, args.perturb_steps,
                                             warmup=args.warmup)
    t_solve = float(np.mean(times))
    value = 1.0 / t_solve
    sample = (f"{len(times)} whole oracle {variant} solves of this workload ({iters} iterations to eps each), "
              f"timed one by one after {args.warmup} untimed ones, as many as fit {args.ref_budget:.0f} s "
              f"of CPU time with the untimed ones")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * t_solve,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(config_of(work, variant, prob, iters, args), parallelism=f"replicas x{world}"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(work, variant, prob, iters, args=None):
    """The workload as both arms name it."""
    c = {"workload": work.name, "variant": variant, "n": work.n, "n_angles": work.n_angles,
         "n_bins": work.n_bins, "eps": prob.eps, "iters": iters, "data_projector": "oracle (FP64)",
         "l2": "flushed (512 MiB write) before each step", "per_gpu_problems": 1}
    if args is not None and args.perturb == "prox" and variant not in ("CG", "PCG", "FISTA"):
        c.update(perturb="prox", prox_iters=args.prox_iters)
    if args is not None and args.perturb_steps > 1 and variant not in ("CG", "PCG", "FISTA"):
        c["perturb_steps"] = args.perturb_steps
    return c


# ---------------------------------------------------------------------------
def run_ours(args, work, rank, local_rank, world):
    import torch
    import torch.distributed as dist

    from paper_1709_04912_gb300 import scg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    scg.load()
    variant = args.variant
    kw = dict(gamma0_rel=args.gamma0_rel, max_iter=work.max_iter, host_loop=int(args.host_loop))
    if variant in ("CG", "PCG"):
        kw["perturb"] = "none"
    elif args.perturb == "prox":
        kw.update(perturb="prox", prox_iters=args.prox_iters)
    if variant not in ("CG", "PCG", "FISTA") and args.perturb_steps > 1:
        kw["perturb_steps"] = args.perturb_steps
    if variant == "FISTA":              # c^2 estimated on the device once, then cached
        kw = dict(lambda_=args.lam, prox_iters=args.prox_iters, max_iter=300, host_loop=int(args.host_loop))

    import oracle
    prob = inputs.make_problem(work, args.seed + rank, oracle.project)
    dtype = DTYPES[args.dtype or "f32"]
    esize = torch.tensor([], dtype=dtype).element_size()
    y = torch.tensor(prob.y, dtype=torch.float32).to(dtype).to(dev)
    out = torch.empty((work.n, work.n), dtype=dtype, device=dev)
    nbytes = scg.solve_workspace_bytes(work.n, work.n_angles, work.n_bins, variant, scg._prec_of(dtype),
                                       **{k: v for k, v in kw.items() if k != "host_loop"})
    wsp = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def solve():
        return scg.scg_solve(y, work.n, variant, prob.eps, out=out, work=wsp, **kw)

    for _ in range(args.warmup):
        r = solve()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms = []
    launches = 0
    results = []
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = solve()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        launches += r.kernel_launches
        results.append(r)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    barrier(world)
    t_total = max_over_ranks(sum(ms) / 1e3, world, dev)
    value = job_rate(args.steps, world, t_total)
    last = results[-1]

    # end to end through the public API with host buffers: pinned y in, x out
    e2e = None
    if not args.no_e2e:
        y_host = torch.tensor(prob.y, dtype=torch.float32).to(dtype).pin_memory()
        x_host = torch.empty((work.n, work.n), dtype=dtype).pin_memory()
        y_dev = torch.empty_like(y)
        t_e2e = 0.0
        for q in range(args.warmup + args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            y_dev.copy_(y_host, non_blocking=True)
            rr = scg.scg_solve(y_dev, work.n, variant, prob.eps, out=out, work=wsp, **kw)
            x_host.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
            if q >= args.warmup:
                t_e2e += time.perf_counter() - t0
        e2e = {"value": args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(y_host.numel() * esize),
               "d2h_bytes_per_step": int(x_host.numel() * esize + 64)}

    # dominant kernels timed alone (CUDA events on the launching stream)
    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    nnz = nnz_of(work)
    xk = out.clone()
    rk = torch.randn((work.n_angles, work.n_bins), dtype=torch.float32, device=dev).to(dtype)

    # the operator pair prepared once (scg_operator_*): each application is
    # device work only -- a one-thread descriptor update, the view (or
    # pair-row) pass and the projector (or backprojector); L2 is flushed
    # before every application and the events bracket the application alone
    op = scg.Operator(work.n, work.n_angles, work.n_bins, dtype, dev, timing=True)

    def time_op(fn, which, reps=20):
        # application time (CUDA events around the call) and the kernel's own
        # device time (events the library records around the kernel alone)
        for _ in range(3):
            fn()
        app, kern = [], []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(1)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            app.append(a.elapsed_time(b))
            kern.append(op.kernel_ms()[which])
        return float(np.mean(kern)), float(np.mean(app))

    yk = torch.empty_like(y)
    gk = torch.empty_like(out)
    t_proj, t_proj_app = time_op(lambda: op.project(xk, yk), 0)
    t_back, t_back_app = time_op(lambda: op.backproject(rk, gk), 1)
    op.close()
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sms * 128 * clock_mhz * 1e6 / 1e12          # T lane-ops/s
    dom = "backproject" if t_back >= t_proj else "project"
    t_dom = max(t_back, t_proj)
    achieved = OPS_PER_NNZ * nnz / (t_dom * 1e-3) / 1e12
    bytes_pass = esize * (work.J + 2 * work.L)
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            import hashlib
            src = open(os.path.join(ROOT, "paper_1709_04912_gb300", "csrc", "kernels.cu"), "rb").read()
            tj = json.load(open(tpath))
            ent = tj.get(f"{dom}:{work.name}")
            if ent and ent.get("kernels_sha1") == hashlib.sha1(src).hexdigest():
                traffic = ent.get("bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    roofline = {"bound": "alu", "kernel": f"k_{dom}",
                "timed_unit": f"k_{dom} alone: CUDA events the library records on the launching stream "
                              "immediately before and after the kernel (scg_operator_kernel_ms), mean of 20 "
                              "applications with the L2 flushed before each",
                "achieved": achieved, "peak": peak_ops,
                "unit": "Top/s (FP32 lane ops)", "frac": achieved / peak_ops, "traffic": traffic,
                "peak_source": f"{sms} SMs x 128 FP32 lanes x {clock_mhz:.0f} MHz ({peak_kind} clock)",
                "ops_per_nnz": OPS_PER_NNZ, "ops_per_launch": OPS_PER_NNZ * nnz, "nnz": nnz,
                "frac_at_min_ops": OPS_PER_NNZ_MIN * nnz / (t_dom * 1e-3) / 1e12 / peak_ops,
                "ms_per_launch": {"project": t_proj, "backproject": t_back},
                "ms_per_application": {"project": t_proj_app, "backproject": t_back_app,
                                       "includes": "1-thread descriptor update + view / pair-row pass + the kernel"},
                "hbm_gbs_algorithmic": {"project": bytes_pass / (t_proj * 1e-3) / 1e9,
                                        "backproject": bytes_pass / (t_back * 1e-3) / 1e9,
                                        "peak": peaks.get("hbm_gbs")},
                # the rate a stored-matrix SpMV would need (8 B per nonzero: value + index)
                # to match this matrix-free pass
                "spmv_equivalent_gbs": {"project": 8 * nnz / (t_proj * 1e-3) / 1e9,
                                        "backproject": 8 * nnz / (t_back * 1e-3) / 1e9}}

    # CPU baseline: whole oracle solves of the same problem, timed
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        times, o_iters, cores = time_oracle_solves(prob, work, variant, args.gamma0_rel, 30.0, 1, args.lam,
                                                   args.prox_iters, args.perturb, args.perturb_steps)
        cpu = {"value": 1.0 / float(np.mean(times)), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"{len(times)} whole oracle {variant} solve(s) of this workload "
                          f"({o_iters} iterations to eps), timed")}

    blocks = {}
    if variant == "FISTA":                      # scg_solve only
        args.no_batch = args.no_serving = True
    if not args.no_batch:
        blocks["batch"] = batch_block(args, dev, rank, world, count=args.batch, dtype_name="f16", steps=3,
                                      warmup=1)
    if not args.no_serving and world == 1:
        blocks["serving"] = serving_block(args, dev, rank, rate=args.rate or 200.0,
                                          duration=args.duration or 8.0, warm=args.serve_warmup or 2.0,
                                          dtype_name="f16")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype or "f32",
                "data": "synthetic",
                "config": dict(config_of(work, variant, prob, last.iters, args), parallelism=f"replicas x{world}"),
                "result": {"status": last.status, "tv_final": last.tv_final, "f_final": last.f_final},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "device_loop": bool(last.device_loop), "clocks": clk,
                "step_ms": ms}
        line.update(blocks)
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def _dtypes():
    import torch
    return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16, "f64": torch.float64}


class _LazyDtypes(dict):
    def __missing__(self, key):
        self.update(_dtypes())
        return dict.__getitem__(self, key)


DTYPES = _LazyDtypes()


def _gpu_problems(works, seed, dev):
    import torch

    from paper_1709_04912_gb300 import scg

    def gpu_project(x, na, nb):
        xt = torch.tensor(x, dtype=torch.float32, device=dev)
        return scg.scg_project(xt, na, nb).double().cpu().numpy()

    probs = [inputs.make_problem(w, seed + q, gpu_project) for q, w in enumerate(works)]
    ys = [torch.tensor(p.y, dtype=torch.float32, device=dev) for p in probs]
    return probs, ys


def _solve_kw(args, variant):
    kw = dict(gamma0_rel=args.gamma0_rel, max_iter=100)
    if variant in ("CG", "PCG"):
        kw["perturb"] = "none"
    return kw


def _same_eps_tv(res, ref, eps):
    """How results of one precision compare with plain-FP32 solo results of the
    same problems: every result within its eps, iteration counts, relative TV
    differences."""
    tv = np.array([abs(a.tv_final - b.tv_final) / max(abs(b.tv_final), 1e-300) for a, b in zip(res, ref)])
    return {"all_f_le_eps": bool(all(r.status == "ok" and r.f_final <= e for r, e in zip(res, eps))),
            "iters_equal": int(sum(a.iters == b.iters for a, b in zip(res, ref))), "problems": len(res),
            "tv_rel_diff_vs_fp32": {"median": float(np.median(tv)), "p95": float(np.percentile(tv, 95)),
                                    "max": float(tv.max()), "within_1pct": int(np.sum(tv <= 0.01))}}


def batch_block(args, dev, rank, world, count, dtype_name, steps, warmup):
    """The uneven batch recipe (N in {128..768}, 60..720 angles, bins
    ceil(sqrt2 N), 1 % noise): ``count`` problems through scg_solve_batch in
    ``dtype_name`` storage, against the same problems one by one through
    scg_solve in that storage and in plain FP32."""
    import torch

    from paper_1709_04912_gb300 import scg

    variant = args.variant
    kw = _solve_kw(args, variant)
    dtype = DTYPES[dtype_name]
    works = inputs.batch_workloads(count, args.seed + rank)
    probs, ys32 = _gpu_problems(works, 1000 * (args.seed + rank), dev)
    ys = [y.to(dtype) for y in ys32]
    ns = [w.n for w in works]
    eps = [p.eps for p in probs]
    outs = [torch.empty((n, n), dtype=dtype, device=dev) for n in ns]
    nbytes = scg.batch_workspace_bytes([(w.n, w.n_angles, w.n_bins) for w in works], variant, dtype)
    wsp = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def batch():
        return scg.scg_solve_batch(ys, ns, variant, eps, outs=outs, work=wsp, **kw)

    for _ in range(warmup):
        rb = batch()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(dev.index)
    clocks.start()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rb = batch()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    barrier(world)
    t_batch = max_over_ranks(float(np.mean(ms)) / 1e3, world, dev)

    def one_by_one(yl, dt):
        w = torch.empty(max(scg.solve_workspace_bytes(wk.n, wk.n_angles, wk.n_bins, variant, scg._prec_of(dt))
                            for wk in works), dtype=torch.uint8, device=dev)
        o = [torch.empty((n, n), dtype=dt, device=dev) for n in ns]
        for q in range(len(works)):                      # warm: one graph per geometry
            scg.scg_solve(yl[q], ns[q], variant, eps[q], out=o[q], work=w, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [scg.scg_solve(yl[q], ns[q], variant, eps[q], out=o[q], work=w, **kw) for q in range(len(works))]
        e1.record(stream)
        e1.synchronize()
        return res, e0.elapsed_time(e1) / 1e3

    solo, t_solo = one_by_one(ys, dtype)
    same = all(a.iters == b.iters and a.tv_final == b.tv_final for a, b in zip(rb, solo))
    fp32_batch = None
    if dtype == torch.float32:
        solo32, t_solo32 = solo, t_solo
    else:
        solo32, t_solo32 = one_by_one(ys32, torch.float32)
        # the same batch in FP32 storage: results bit-identical to the FP32 solo solves
        nb32 = scg.batch_workspace_bytes([(w.n, w.n_angles, w.n_bins) for w in works], variant, torch.float32)
        wsp32 = torch.empty(nb32, dtype=torch.uint8, device=dev)
        o32 = [torch.empty((n, n), dtype=torch.float32, device=dev) for n in ns]
        r32 = scg.scg_solve_batch(ys32, ns, variant, eps, outs=o32, work=wsp32, **kw)
        torch.cuda.synchronize()
        ms32 = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r32 = scg.scg_solve_batch(ys32, ns, variant, eps, outs=o32, work=wsp32, **kw)
            e1.record(stream)
            e1.synchronize()
            ms32.append(e0.elapsed_time(e1))
        t32 = max_over_ranks(float(np.mean(ms32)) / 1e3, world, dev)
        fp32_batch = {"value": job_rate(len(works), world, t32), "unit": UNIT, "ms_per_batch": 1e3 * t32,
                      "speedup_vs_fp32_solo": t_solo32 / t32,
                      "same_iters_and_tv_as_fp32_solo": bool(all(a.iters == b.iters and a.tv_final == b.tv_final
                                                                 for a, b in zip(r32, solo32)))}
        del wsp32
    value = job_rate(len(works), world, t_batch)
    return {"metric": "batched recon/s", "value": value, "unit": UNIT, "dtype": dtype_name,
            "ms_per_batch": 1e3 * t_batch, "steps": steps, "warmup": warmup, "step_ms": ms,
            "config": {"workload": f"uneven_batch{len(works)}", "variant": variant,
                       "sizes": "N in {128,...,768}, angles in {60,...,720}, bins ceil(sqrt2 N), 1 % noise",
                       "data_projector": "libscg FP32", "workspace_bytes": nbytes,
                       "total_iters": int(sum(r.iters for r in rb)), "body_launches": rb[0].body_launches},
            "solo_same_storage": {"value": len(works) / t_solo, "unit": UNIT, "same_iters_and_tv": bool(same)},
            "solo_fp32": {"value": len(works) / t_solo32, "unit": UNIT},
            "speedup_vs_fp32_solo": t_solo32 / t_batch,
            "equal_eps_and_tv": _same_eps_tv(rb, solo32, eps), "fp32_batch": fp32_batch, "clocks": clk}


def serving_block(args, dev, rank, rate, duration, warm, dtype_name):
    """A Poisson stream of few-view requests (N ~ U{128..1024 step 64}, 30..180
    angles, eps factor U[1.02, 1.2], 1 % noise) through the continuous-batching
    server; latency is arrival to completion on the host clock.  Also the
    saturated rate (128 requests queued at once) and the same requests solved
    one by one on the plain FP32 single-solve path."""
    import torch

    from paper_1709_04912_gb300 import scg

    variant = args.variant
    kw = _solve_kw(args, variant)
    dtype = DTYPES[dtype_name]
    uniq = inputs.serving_workloads(64, args.seed + rank)
    probs, ys32 = _gpu_problems(uniq, 5000 * (args.seed + rank), dev)
    ys = [y.to(dtype) for y in ys32]
    outs = [torch.empty((w.n, w.n), dtype=dtype, device=dev) for w in uniq]
    srv = scg.Server(variant, dtype, pool_bytes=int(args.pool_gb * (1 << 30)), max_active=args.max_active,
                     device=dev, **kw)

    def submit(q, tag):
        u = q % len(uniq)
        srv.submit(ys[u], uniq[u].n, probs[u].eps, out=outs[u], tag=tag)

    sat = []
    served = {}
    for _ in range(2):                                   # the first pass also captures the graphs
        t0 = time.perf_counter()
        for q in range(2 * len(uniq)):
            submit(q, q)
        got = 0
        while got < 2 * len(uniq):
            for tag, r in srv.step():
                served[tag % len(uniq)] = r
                got += 1
        sat.append(2 * len(uniq) / (time.perf_counter() - t0))
    wsolo = torch.empty(max(scg.solve_workspace_bytes(w.n, w.n_angles, w.n_bins, variant, scg.F32)
                            for w in uniq), dtype=torch.uint8, device=dev)
    o32 = [torch.empty((w.n, w.n), dtype=torch.float32, device=dev) for w in uniq]
    for q in range(len(uniq)):
        scg.scg_solve(ys32[q], uniq[q].n, variant, probs[q].eps, out=o32[q], work=wsolo, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solo_res = [scg.scg_solve(ys32[q], uniq[q].n, variant, probs[q].eps, out=o32[q], work=wsolo, **kw)
                for q in range(len(uniq))]
    torch.cuda.synchronize()
    solo = len(uniq) / (time.perf_counter() - t0)
    same = _same_eps_tv([served[q] for q in range(len(uniq))], solo_res, [p.eps for p in probs])
    total = warm + duration
    arrivals = inputs.poisson_arrivals(int(rate * total * 1.5) + 16, rate, args.seed + 7)
    arrivals = arrivals[arrivals < total]
    lat, done_t = {}, {}
    clocks = ClockSampler(dev.index)
    clocks.start()
    t_start = time.perf_counter()
    nxt = 0
    steps = 0
    while True:
        now = time.perf_counter() - t_start
        while nxt < len(arrivals) and arrivals[nxt] <= now:
            submit(nxt, 100000 + nxt)
            nxt += 1
        queued, active = srv.pending()
        if queued == 0 and active == 0:
            if nxt >= len(arrivals):
                break
            time.sleep(max(0.0, min(arrivals[nxt] - now, 0.01)))
            continue
        for tag, r in srv.step():
            q = tag - 100000
            t = time.perf_counter() - t_start
            done_t[q] = t
            lat[q] = t - arrivals[q]
        steps += 1
    clk = clocks.stop()
    srv.close()
    window = [q for q in lat if warm <= arrivals[q] < total]
    L = np.array([lat[q] for q in window]) * 1e3 if window else np.array([float("nan")])
    t_end = max(done_t[q] for q in window) if window else total
    thr = len(window) / max(t_end - warm, 1e-9)
    return {"metric": "served recon/s (Poisson)", "value": thr, "unit": UNIT, "dtype": dtype_name,
            "steps": steps,
            "config": {"workload": "serving_poisson", "variant": variant, "rate": rate, "duration_s": duration,
                       "warmup_s": warm, "requests": len(window), "max_active": args.max_active,
                       "pool_gb": args.pool_gb, "data_projector": "libscg FP32",
                       "sizes": "N ~ U{128..1024 step 64}, 30..180 angles, eps 1.02-1.2 x noise floor"},
            "latency_ms": {"p50": float(np.percentile(L, 50)), "p99": float(np.percentile(L, 99)),
                           "mean": float(np.mean(L))},
            "saturated_recon_per_s": max(sat), "solo_fp32_recon_per_s": solo,
            "saturated_vs_fp32_solo": max(sat) / solo, "equal_eps_and_tv": same, "clocks": clk}


def run_batch(args, rank, local_rank, world):
    """--mode batch: the batch block alone, as its own line."""
    import torch

    from paper_1709_04912_gb300 import scg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    scg.load()
    b = batch_block(args, dev, rank, world, args.batch, args.dtype or "f32", args.steps, args.warmup)
    if rank == 0:
        line = dict(b, n_gpus=world, higher_is_better=True, scaling="weak", vs_baseline=None, data="synthetic")
        line["config"]["parallelism"] = f"replicas x{world}"
        print(json.dumps(line), flush=True)
    return 0


def run_serving(args, rank, local_rank, world):
    """--mode serving: the serving block alone, as its own line."""
    import torch

    from paper_1709_04912_gb300 import scg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    scg.load()
    b = serving_block(args, dev, rank, args.rate or 50.0, args.duration or 20.0, args.serve_warmup or 5.0,
                      args.dtype or "f16")
    if rank == 0:
        line = dict(b, n_gpus=world, warmup=0, ms_per_step=None, higher_is_better=True, scaling="weak",
                    vs_baseline=None, data="synthetic")
        line["value"] = b["value"] * world
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, local_rank, world = dist_env()
    work = WORKLOADS[args.workload]
    if world > 1:
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return 0
        else:
            import torch
            torch.cuda.set_device(local_rank)          # each rank's collectives on its own GPU
            dist.init_process_group("nccl", init_method="env://")
    if args.impl == "reference":
        return run_reference(args, work, rank, world)
    if args.mode == "batch":
        return run_batch(args, rank, local_rank, world)
    if args.mode == "serving":
        return run_serving(args, rank, local_rank, world)
    return run_ours(args, work, rank, local_rank, world)


if __name__ == "__main__":
    sys.exit(main())
