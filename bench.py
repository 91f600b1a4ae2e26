"""Benchmark of the two-site DMRG hot path on GB300.

One step = one full two-site update at the central bond of the K=40, N=40,
S_z=0, M=2000 workload (the configuration the headline metric is quoted on):
W-contracted operators, diagonal of H_eff, Davidson with a fixed iteration
budget (16 by default, about what sweeps take per site; each iteration one
H_eff.psi), decimation to M states and the environment update of the new bond.
The default arithmetic is the one that meets the metric's accuracy: H_eff.psi on
the tensor cores with three BF16 slices on the TMA-staged work lists (precision 5)
and the environment update on the tensor cores with exactly split operands
(environment precision 3, FP64-level results).  Inputs (integrals, a random QN-block MPS
with bond dimension 2000 and its environments, tens of GB) are built before
the timed region and stay resident in HBM; they are far larger than L2, so no
explicit flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the hot path of one problem is not sharded here (replicas only):
each rank runs its own replica of the workload on its own GPU, value is the
sum over ranks, time the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H_eff·ψ TFLOP/s & sweep s at K=40 M=2000, mixed vs FP64 GPU at |ΔE|≤1e-6 Eh"
# DRAM bytes (read + write) of one H_eff.psi of the K=40 centre workload, both stages,
# per precision, from one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum
# (profiles/gemm_tma_kernel_sigma_k40_m2000.md); absent where not captured for the
# current kernels
TRAFFIC = {5: 26.46e9 + 37.16e9 + 66.38e9 + 0.05e9, 4: 8.20e9 + 12.29e9 + 21.40e9 + 0.04e9}

WORKLOADS = {
    # name: K, N, two_sz, M, spread of the synthetic sector dimensions, integral seed, h off-diagonal std,
    # M schedule of a full run (--sweeps), starting bond dimension of the random MPS
    "k40_m2000": dict(K=40, N=40, two_sz=0, M=2000, spread=1.0, seed=1607, offdiag_std=0.05,
                      ramp=[250, 500, 1000, 2000, 2000, 2000], m0=250),
    "k24_m512": dict(K=24, N=24, two_sz=0, M=512, spread=1.0, seed=1606, offdiag_std=0.1,
                     ramp=[128, 256] + [512] * 8, m0=128),
    "k32_m1024": dict(K=32, N=32, two_sz=0, M=1024, spread=1.0, seed=1609, offdiag_std=0.1,
                      ramp=[128, 256, 512, 1024, 1024, 1024], m0=128),
    "k16_m256": dict(K=16, N=16, two_sz=0, M=256, spread=1.0, seed=1606, offdiag_std=0.1,
                     ramp=[64, 128, 256, 256], m0=64),
}
# bounded CPU sample for the oracle: the projected-H_eff oracle works in the
# full Fock space, so it can only take K <= 10; this is the largest sample of
# the same kind of step (central two-site sigma) it finishes in seconds
ORACLE_SAMPLE = dict(K=10, N=10, two_sz=0, M=1000, k=3, seed=1607, spread=0.5)
# Algorithmic flops of one H_eff.psi of that sample: the sum of 2mnk over the non-zero
# quantum-number blocks of the MPO contraction (the count every TFLOP/s figure here
# uses).  The oracle builds no MPO, so it cannot count them itself; the value is
# stored so that the oracle arm runs without the CUDA library, and
# tests/test_bench_contract.py checks it against the library's host-side count.
ORACLE_SAMPLE_FLOPS = 2928679808.0


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

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
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(seconds: float = 12.0):
    """Time the CPU oracle's sigma (P^T H P psi) on the bounded sample; returns
    (sigma flops of the sample, seconds per sigma, calls)."""
    from oracle import mps as omps
    from paper_1605_02611_gb300 import synth
    s = ORACLE_SAMPLE
    h, eri = synth.integrals(s["K"], s["seed"])
    bonds, T = synth.random_mps(s["K"], s["N"], s["two_sz"], s["M"], s["seed"] + 1, s["spread"])
    k = s["k"]
    psi = synth.random_psi(bonds[k], bonds[k + 2], s["seed"] + 2)
    Na = Nb = s["N"] // 2
    flops = ORACLE_SAMPLE_FLOPS
    P = omps.TwoSiteProjector(T, k, Na, Nb)
    omps.sigma(T, k, psi, h, eri, Na, Nb, P)  # warm-up (string tables)
    t0 = time.perf_counter()
    n = 0
    while True:
        omps.sigma(T, k, psi, h, eri, Na, Nb, P)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = (time.perf_counter() - t0) / n
    return flops, dt, n


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max((x.get("num_threads") or 0) for x in threadpool_info()) or os.cpu_count()
    except Exception:
        return os.cpu_count()


def dgemm_measured(torch):
    """cuBLAS FP64 GEMM throughput on this GPU (context for the FP64 roofline)."""
    n = 4096
    a = torch.randn(n, n, device="cuda", dtype=torch.float64)
    b = torch.randn(n, n, device="cuda", dtype=torch.float64)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2 * n ** 3 / best / 1e9


def workload_name(args, sigma_calls_per_step=None):
    """The workload both arms report: the central two-site step of the named workload."""
    w = WORKLOADS[args.workload]
    K = w["K"]
    k = K // 2 - 1
    ref = f", refinement by precision {args.refine} ({args.refine_iters} of the iterations)" if args.refine >= 0 else ""
    env = {0: ", FP64 environment update", 2: ", tensor-core environment update (three BF16 slices)",
           3: ", tensor-core environment update (exactly split operands)"}[args.env_precision]
    meas = f", {sigma_calls_per_step:.1f} sigma calls/step measured" if sigma_calls_per_step is not None else ""
    return (f"{args.workload}: K={K} N={w['N']} 2Sz={w['two_sz']} M={w['M']}, two-site step at sites "
            f"({k},{k + 1}), Davidson budget {args.dav_iters} iterations/step{meas}, precision {args.precision}"
            f"{ref}{env}")


def aggregate_ranks(ms, flops, t_e2e, e2e_flops, world, device):
    """Whole-job figures over the replicas: times are the maximum over ranks,
    flops the sum (every rank runs its own replica of the workload)."""
    if world <= 1:
        return ms, flops, t_e2e, e2e_flops
    import torch
    t = torch.tensor([ms, flops, t_e2e, e2e_flops], dtype=torch.float64, device=device)
    mx = t.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    sm = t.clone()
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(mx[2]), float(sm[3])


def run_reference(args, rank, world):
    """Oracle arm: the CPU oracle on a bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return
    times = []
    flops = None
    for i in range(args.warmup + args.steps):
        fl, dt, n = oracle_sample(seconds=3.0)
        flops = fl
        if i >= args.warmup:
            times.append(dt)
    dt = sum(times) / len(times)
    value = flops / dt / 1e12
    cores = blas_threads()
    sample = (f"oracle sigma (P^T H P psi via direct CI) at K={ORACLE_SAMPLE['K']}, M={ORACLE_SAMPLE['M']}, "
              f"sites ({ORACLE_SAMPLE['k']},{ORACLE_SAMPLE['k'] + 1}); the oracle cannot hold K=40")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "parallelism": f"replicas{world}", "sample": sample},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1605_02611_gb300 as G
    from paper_1605_02611_gb300 import synth

    torch.cuda.set_device(local_rank)
    w = WORKLOADS[args.workload]
    K, N, M = w["K"], w["N"], w["M"]
    k = K // 2 - 1
    t_setup = time.perf_counter()
    h, eri = synth.integrals(K, w["seed"], w["offdiag_std"])
    bonds, T = synth.random_isometric_mps(K, N, w["two_sz"], M, w["seed"] + 1, k, w["spread"])
    stream = torch.cuda.Stream()
    ctx = G.Context(h, eri, N, w["two_sz"], stream=stream.cuda_stream)
    ctx.set_precision(args.precision)
    if args.stage1_stacked:
        ctx.set_stage1_stacked(True)
    if args.fp64_w_sums:
        ctx.set_tc_combos(False)
    if args.env_precision:
        ctx.set_env_precision(args.env_precision)
    if args.refine >= 0:
        ctx.set_refinement(args.refine, args.refine_iters)
    ctx.set_mps(T, [b.labels() for b in bonds])
    del T
    # should the tensor-core W-contracted sums report an error (here or in the first
    # warm-up step), the run continues with FP64 sums and says so in the line
    w_sums_failed = None

    def with_fp64_fallback(fn):
        nonlocal w_sums_failed
        try:
            return fn()
        except G.GbdmrgError as exc:
            # only the errors the tensor-core sums report on purpose (an operator class
            # too large for them, a bounded wait that ran out, no memory for their
            # operands); a CUDA fault or anything else ends the run
            if args.fp64_w_sums or w_sums_failed is not None or exc.status not in ("EINVAL", "ETIMEOUT", "ENOMEM"):
                raise
            w_sums_failed = str(exc)
            print(f"warning: tensor-core W-contracted sums failed, using FP64 sums: {exc}", file=sys.stderr)
            ctx.set_tc_combos(False)
            ctx.prepare(k)
            return fn()

    with_fp64_fallback(lambda: ctx.prepare(k))
    nnz = ctx.nnz
    plan_stats = ctx.plan_stats() if args.precision >= 4 else None
    setup_s = time.perf_counter() - t_setup
    setup_launches = G.kernel_launches()
    dav = args.dav_iters
    if args.profile_sigma:
        # profiling helper: only H_eff.psi calls on device buffers, then exit
        x = torch.randn(nnz, device="cuda", dtype=torch.float64)
        y = torch.empty_like(x)
        for _ in range(args.profile_sigma):
            ctx.sigma_device(x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        print(json.dumps({"profile_sigma": args.profile_sigma, "setup_launches": setup_launches, "psi_nnz": nnz}))
        ctx.close()
        return

    def step(psi_in=None, want=False):
        return ctx.step(k, 0, M, 1e-14, dav, psi_in=psi_in, want_psi=want)

    with_fp64_fallback(step)
    for _ in range(args.warmup - 1):
        step()
    torch.cuda.synchronize()
    c0 = ctx.counters()
    p0 = ctx.phase_times()
    pf0 = ctx.phase_flops()
    l0 = G.kernel_launches()
    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if args.profiler_range:
        torch.cuda.cudart().cudaProfilerStart()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if args.profiler_range:
        torch.cuda.cudart().cudaProfilerStop()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    c1 = ctx.counters()
    p1 = ctx.phase_times()
    pf1 = ctx.phase_flops()
    phases = {kk: round((p1[kk] - p0[kk]) / args.steps, 4) for kk in p1}
    phase_tf = {kk: round((pf1[kk] - pf0[kk]) / max(p1[kk] - p0[kk], 1e-12) / 1e12, 3) for kk in p1}
    launches = G.kernel_launches() - l0
    flops = (c1["sigma_flops"] - c0["sigma_flops"]) + (c1["other_flops"] - c0["other_flops"])
    sig_fl = c1["sigma_flops"] - c0["sigma_flops"]
    sig_s = c1["sigma_seconds"] - c0["sigma_seconds"]
    sig_calls = c1["sigma_calls"] - c0["sigma_calls"]
    # end to end through the public API with host buffers: psi in / optimised psi out
    psi_host = np.zeros(nnz)
    _, _, _, psi_host = step(want=True)
    torch.cuda.synchronize()
    ce0 = ctx.counters()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, _, _, out = step(psi_in=psi_host, want=True)
    t_e2e = time.perf_counter() - t0
    ce1 = ctx.counters()
    e2e_flops = (ce1["sigma_flops"] - ce0["sigma_flops"]) + (ce1["other_flops"] - ce0["other_flops"])

    ms, flops, t_e2e, e2e_flops = aggregate_ranks(ms, flops, t_e2e, e2e_flops, world, "cuda")
    if rank != 0:
        return
    value = flops / (ms * 1e-3) / 1e12
    peaks, src = _measured_peaks()
    achieved_alg = sig_fl / sig_s / 1e12 if sig_s > 0 else None
    # The sigma kernels of the step timed on their own after the timed region (CUDA
    # events on the context stream, inputs resident in HBM, larger than L2): the
    # step's operator and, with refinement, the refinement operator.
    kern = {}
    xk = torch.randn(nnz, device="cuda", dtype=torch.float64)
    yk = torch.empty_like(xk)
    torch.cuda.synchronize()
    for label, prec in (("primary", args.precision), ("refine", args.refine)):
        if prec is None or prec < 0 or (label == "refine" and prec == args.precision):
            continue
        ctx.set_precision(prec)
        ctx.plan(k)
        flk = ctx.sigma_device(xk.data_ptr(), yk.data_ptr())
        msk = ctx.sigma_timing(3, xk.data_ptr(), yk.data_ptr())
        kern[label] = {"precision": prec, "ms": msk, "tflops": flk / msk / 1e9,
                       "plan": ctx.plan_stats() if prec >= 4 else None}
    ctx.set_precision(args.precision)
    # products the tensor cores execute per algorithmic multiply-add: 1 (one BF16
    # pass) or 6 (three BF16 slices, products s_i t_j with i + j <= 2)
    nprod = {0: 1, 1: 1, 2: 6, 3: 3, 4: 1, 5: 6, 6: 3}[args.precision]
    fp64_cmp = None
    if args.precision > 0 and args.compare_fp64:
        # full-size checks (outside the timed region): the tensor-core H_eff.psi of the
        # bench's own work lists against the FP64 one on the same vector, and the
        # Hermiticity <x2|H x> = <H x2|x> of the FP64 operator
        checks = {}
        x = torch.randn(nnz, device="cuda", dtype=torch.float64)
        x2 = torch.randn(nnz, device="cuda", dtype=torch.float64)
        y, y2, y_tc = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        torch.cuda.synchronize()
        try:
            ctx.plan(k)
            ctx.sigma_device(x.data_ptr(), y_tc.data_ptr())
        except Exception as exc:  # reported in the line, never fatal for the bench
            checks["error"] = f"tensor-core sigma: {exc}"
        # the same H_eff.psi on the FP64 units (one call), for the mixed/FP64 speed-up;
        # the W-contracted sums are rebuilt on the FP64 units too, so the comparison is
        # against an operator formed entirely in FP64
        ctx.set_precision(0)
        ctx.set_tc_combos(False)
        ctx.plan(k)
        fl64 = ctx.sigma_device(x.data_ptr(), y.data_ptr())
        ms64 = ctx.sigma_timing(1, x.data_ptr(), y.data_ptr())
        fp64_cmp = {"sigma_ms": ms64, "sigma_tflops": fl64 / ms64 / 1e9,
                    "speedup_mixed_over_fp64": (fl64 / ms64 / 1e9) and (achieved_alg / (fl64 / ms64 / 1e9))}
        try:
            ctx.sigma_device(x2.data_ptr(), y2.data_ptr())
            ny = float(torch.linalg.vector_norm(y))
            if "error" not in checks:
                checks["sigma_rel_err_vs_fp64"] = float(torch.linalg.vector_norm(y_tc - y)) / ny
                checks["sigma_max_rel_err_vs_fp64"] = float((y_tc - y).abs().max()) / float(y.abs().max())
            x2_hx, hx2_x = float(torch.dot(x2, y)), float(torch.dot(y2, x))
            checks["fp64_hermiticity"] = abs(x2_hx - hx2_x) / (float(torch.linalg.vector_norm(x2)) * ny)
        except Exception as exc:
            checks["error"] = f"fp64 checks: {exc}"
        fp64_cmp["fullsize_checks"] = checks
    ach_k = kern["primary"]["tflops"]
    if args.precision == 0:
        peak = peaks["bf16_tflops_sustained"] * 1.25 / 2250.0
        roof = {"bound": "alu", "achieved": ach_k, "peak": peak, "unit": "TFLOP/s",
                "frac": ach_k / peak, "traffic": None,
                "kernel": "gemm_f64_kernel (sigma stages 1+2)",
                "peak_note": f"FP64 = {src} bf16 sustained x 1.25/2250 (nominal FP64/BF16)"}
        dtype = "f64"
    else:
        peak = peaks["bf16_tflops_sustained"]
        # achieved = ALGORITHMIC flops (2mnk over non-zero blocks, no padding, no extra
        # split-precision products) / event-timed sigma time; the products the tensor
        # cores actually execute for the slices are reported beside it, not in frac
        roof = {"bound": "tensor", "achieved": ach_k, "peak": peak, "unit": "TFLOP/s",
                "frac": ach_k / peak, "traffic": TRAFFIC.get(args.precision) if args.workload == "k40_m2000" else None,
                "kernel": ("gemm_tma_kernel<1>+<2> (sigma stages 1+2, TMA-staged)" if args.precision >= 4 else
                           "gemm_bf16_tc_kernel (sigma stages 1+2)") + f", precision {args.precision}",
                "executed_tflops": ach_k * nprod,
                "products_per_multiply_add": nprod,
                "peak_note": f"{src} bf16 dense, sustained (kernel timed inside a long step); achieved and frac "
                             f"count algorithmic flops only"}
        dtype = {1: "bf16", 2: "bf16x3", 3: "bf16x2", 4: "bf16", 5: "bf16x3", 6: "bf16x2"}[args.precision]
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": workload_name(args, sig_calls / args.steps),
                   "psi_nnz": nnz, "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (no flush)",
                   "setup_s": round(setup_s, 1), "setup_launches": int(setup_launches),
                   "stage1": "stacked" if args.stage1_stacked else "per-sector",
                   "w_sums": "fp64" if args.fp64_w_sums else
                   (f"fp64 (tensor-core sums failed: {w_sums_failed})" if w_sums_failed else
                    "tensor cores (bf16x3) for sums of >= 1e5 terms that feed only the sigma, fp64 otherwise")},
        "sigma_tflops": achieved_alg, "sigma_calls": sig_calls, "sigma_kernels": kern, "fp64_comparison": fp64_cmp,
        "tma_plan": plan_stats,
        "step_phase_s": phases,
        "step_phase_tflops": phase_tf,
        "roofline": roof,
        "e2e": {"value": e2e_flops / t_e2e / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": nnz * 8,
                "d2h_bytes_per_step": nnz * 8},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        fl, dt, n = oracle_sample(seconds=args.cpu_seconds)
        line["cpu_baseline"] = {
            "value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": blas_threads(), "kind": "oracle",
            "sample": f"{n} oracle sigmas (P^T H P psi, direct CI) at K={ORACLE_SAMPLE['K']}, "
                      f"M={ORACLE_SAMPLE['M']}; the oracle works in the 4^K Fock space and cannot hold K=40"}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_sweeps(args):
    """Full two-site DMRG with the workload's M ramp (the 'sweep s' part of the metric)."""
    import torch

    import paper_1605_02611_gb300 as G
    from paper_1605_02611_gb300 import synth
    w = WORKLOADS[args.workload]
    K, N = w["K"], w["N"]
    ramp = w["ramp"][:args.sweeps] if args.sweeps > 0 else w["ramp"]
    h, eri = synth.integrals(K, w["seed"], w["offdiag_std"])
    bonds, T = synth.random_mps(K, N, w["two_sz"], w["m0"], w["seed"] + 1, w["spread"])
    ctx = G.Context(h, eri, N, w["two_sz"])
    if args.env_precision:
        ctx.set_env_precision(args.env_precision)
    if args.refine >= 0:
        ctx.set_refinement(args.refine, args.refine_iters)
    ctx.set_mps(T, [b.labels() for b in bonds])
    del T
    tol = [1e-5] * (len(ramp) - 1) + [1e-6]
    t0 = time.perf_counter()
    out = ctx.run(ramp, tol, max_iter=args.max_iter, precision=args.precision)
    wall = time.perf_counter() - t0
    c = ctx.counters()
    line = {"mode": "sweeps", "workload": args.workload, "K": K, "N": N, "precision": args.precision,
            "refine": args.refine, "env_precision": args.env_precision,
            "M": ramp, "energy": out["energy"].tolist(), "discarded": out["discarded"].tolist(),
            "sweep_s": out["seconds"].tolist(), "davidson_iters": out["davidson_iters"].tolist(),
            "sigma_tflops": [f / s / 1e12 if s > 0 else None for f, s in zip(out["sigma_flops"], out["sigma_seconds"])],
            "wall_s": wall, "phase_s": ctx.phase_times(), "sigma_calls": c["sigma_calls"]}
    print(json.dumps(line), flush=True)
    ctx.close()


BATCH = dict(P=64, K=(16, 32), M=(256, 1000), seed=4096, spread=1.0)


def run_batched(args):
    """Batched H_eff.psi: P independent central two-site problems (each its own
    integrals, K and M drawn uniformly, half filling, S_z=0) whose tensor-core
    work lists are fused into one persistent launch per stage and replayed as a
    CUDA graph; compared with the same problems' sigmas run one by one."""
    import concurrent.futures as cf

    import torch

    import paper_1605_02611_gb300 as G
    from paper_1605_02611_gb300 import synth
    b = dict(BATCH)
    b["P"] = args.batched
    prec = args.precision if args.precision > 0 else 2
    rng = np.random.default_rng(b["seed"])
    specs = []
    for p in range(b["P"]):
        K = 2 * int(rng.integers(b["K"][0] // 2, b["K"][1] // 2 + 1))
        M = int(rng.integers(b["M"][0], b["M"][1] + 1))
        specs.append((p, K, M))
    torch.cuda.init()

    def build(spec):
        p, K, M = spec
        k = K // 2 - 1
        h, eri = synth.integrals(K, b["seed"] + p)
        bonds, T = synth.random_isometric_mps(K, K, 0, M, b["seed"] + 1000 + p, k, b["spread"])
        ctx = G.Context(h, eri, K, 0)
        ctx.set_precision(prec)
        ctx.keep_host_plans(True)
        ctx.set_mps(T, [bd.labels() for bd in bonds])
        del T
        ctx.prepare(k)
        return ctx

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        ctxs = list(ex.map(build, specs))
    setup_s = time.perf_counter() - t0
    xs = [torch.randn(c.nnz, device="cuda", dtype=torch.float64) for c in ctxs]
    ys = [torch.empty_like(x) for x in xs]
    torch.cuda.synchronize()
    xp = [x.data_ptr() for x in xs]
    yp = [y.data_ptr() for y in ys]
    # the same sigmas one by one (each context on its own stream, in sequence)
    seq_ms = 0.0
    for c, x, y in zip(ctxs, xp, yp):
        c.sigma_device(x, y)
        seq_ms += c.sigma_timing(1, x, y)
    tune = None
    if args.autotune:
        # split-K granularity of the fused work lists, chosen by timing the batched launch
        t_ms, t_split, t_budget = G.autotune(ctxs, reps=3)
        tune = {"split_tiles_per_sm": t_split, "chunk_budget_mb": t_budget,
                "candidates": [32, 8, 2, 0.5, 0.125, 0.03125, 0], "ms": [float(v) for v in t_ms[:, 0]]}
    bt = G.Batch(ctxs)
    eager = []
    fl = 0.0
    for _ in range(args.warmup + args.steps):
        ms, fl = bt.sigma(xp, yp, use_graph=False)
        eager.append(ms)
    bt.sigma(xp, yp, use_graph=True)  # eager pass + capture
    graph = []
    l0 = G.kernel_launches()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for i in range(args.warmup + args.steps):
        ms, fl = bt.sigma(xp, yp, use_graph=True)
        if i >= args.warmup:
            graph.append(ms)
    clk = clocks.stop()
    launches = G.kernel_launches() - l0
    eager_ms = statistics.mean(eager[args.warmup:])
    graph_ms = statistics.mean(graph)
    peaks, src = _measured_peaks()
    nprod = {1: 1, 2: 6, 3: 3}[prec]
    line = {"mode": "batched", "problems": b["P"], "K_range": b["K"], "M_range": b["M"], "precision": prec,
            "Ks": [s[1] for s in specs], "Ms": [s[2] for s in specs], "psi_nnz_total": int(sum(c.nnz for c in ctxs)),
            "flops_per_batch": fl, "sequential_ms": seq_ms, "batched_eager_ms": eager_ms, "batched_graph_ms": graph_ms,
            "sequential_tflops": fl / seq_ms / 1e9, "batched_tflops": fl / graph_ms / 1e9,
            "speedup_over_sequential": seq_ms / graph_ms,
            "tensor_frac": fl / graph_ms / 1e9 / peaks["bf16_tflops_sustained"],
            "executed_tensor_frac": fl * nprod / graph_ms / 1e9 / peaks["bf16_tflops_sustained"],
            "peak_note": f"{src} bf16 sustained; tensor_frac counts algorithmic flops, executed_tensor_frac the "
                         f"{nprod} tensor-core products per algorithmic multiply-add",
            "gpu_launches_per_batch": launches / max(1, args.warmup + args.steps), "setup_s": setup_s,
            "autotune": tune, "clocks": clk}
    print(json.dumps(line), flush=True)
    bt.close()
    for c in ctxs:
        c.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="k40_m2000", choices=sorted(WORKLOADS))
    ap.add_argument("--dav-iters", type=int, default=16,
                    help="Davidson iterations per step (sweeps at K=24 averaged ~20 per site)")
    ap.add_argument("--precision", type=int, default=5, choices=[0, 1, 2, 3, 4, 5, 6],
                    help="0 FP64 units, 1 tensor cores one BF16 pass, 2 tensor cores three BF16 slices, 3 two slices, "
                         "4, 5, 6 one pass, three and two slices on the TMA-staged work lists")
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps", type=int, default=-1,
                    help=">= 0: run a full DMRG with the workload's M ramp (0 = whole ramp) instead of the step bench")
    ap.add_argument("--max-iter", type=int, default=40)
    ap.add_argument("--batched", type=int, default=0,
                    help="> 0: batched H_eff.psi over this many independent problems instead of the step bench")
    ap.add_argument("--stage1-stacked", action="store_true",
                    help="tensor-core sigma with stacked right operands in stage 1")
    ap.add_argument("--fp64-w-sums", action="store_true",
                    help="form every W-contracted sum on the FP64 units (default: large sums that feed only "
                         "the tensor-core sigma run on the tensor cores)")
    ap.add_argument("--env-precision", type=int, default=3, choices=[0, 2, 3],
                    help="environment updates: 0 FP64 units, 2 tensor cores with three BF16 slices, "
                         "3 tensor cores with exactly split operands")
    ap.add_argument("--refine", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4, 5, 6],
                    help="precision of the Davidson refinement phase of each step (-1: none)")
    ap.add_argument("--refine-iters", type=int, default=4,
                    help="Davidson iterations of the step budget given to the refinement phase")
    ap.add_argument("--autotune", action="store_true",
                    help="with --batched: choose the split-K granularity of the fused work lists by timing")
    ap.add_argument("--profiler-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--profile-sigma", type=int, default=0,
                    help="after setup run this many H_eff.psi calls only (for ncu captures) and exit")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.sweeps >= 0:
        if rank == 0:
            run_sweeps(args)
        return
    if args.batched > 0:
        if rank == 0:
            run_batched(args)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
