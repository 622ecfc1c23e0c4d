"""Benchmark of the FOT hot path on GB300: FOT Mpixel*iter/s at 1024^2.

One step = one whole solve of the benchmark workload through the C ABI: problem load
(a = g^2/sum g^2, logs), 200 Sinkhorn iterations (Eqs. 7-8, 4 axis passes each) and the
phase step (moments of Eqs. 9-10 + trapezoid integration).  Workload: 1024 x 1024
two-Gaussian input beam -> seeded composite of 12 flat-top rectangles / disks / rings at
30% coverage, fixed eps = 2e-4 n^2 px^2 (the paper's working eps), 200 iterations.
Inputs are synthetic (seeded); they stand in for the paper's Fig. 1 images.

Prints ONE JSON line (rank 0).  Under torchrun every rank solves its own copy of the
workload (independent problems, no collective on the data path): weak scaling.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FOT Mpixel*iter/s at 1024^2 (mixed vs FP32, <=1e-4 marginal L1); % of roofline"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="fot", choices=["fot", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp32", "fp32_dense", "mixed", "bf16"])
    p.add_argument("--no-compare", action="store_true",
                   help="skip the FP32 comparison run of the mixed form")
    p.add_argument("--n", type=int, default=1024)
    p.add_argument("--iters", type=int, default=200)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-sub", action="store_true",
                   help="skip the sub-records of the single workload (2048^2, the 64-problem batch, "
                        "iterations and time to a 1e-4 marginal violation)")
    p.add_argument("--workload", default="single", choices=["single", "batched", "stopping", "intensity", "cfot", "sweep"],
                   help="batched: the 64-problem uneven-size batch (one graph launch per solve) "
                        "against looping single solves of the same problems; stopping: the "
                        "single workload solved to a marginal-violation tolerance; intensity: the "
                        "L1 intensity loss of that workload's phase; cfot: cFOT against FOT per "
                        "iteration on beams over a flat floor")
    p.add_argument("--cfot-eps", type=float, default=1e5, help="cfot workload: eps in px^2")
    p.add_argument("--tol", type=float, default=0.2,
                   help="stopping workload: tolerance on sum |Gamma 1 - a|")
    p.add_argument("--check-every", type=int, default=10,
                   help="stopping workload: iterations between violation checks")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _config(w, n, a, ws):
    """The workload description both arms print."""
    return {"workload": w.name, "n": n, "iters_per_solve": a.iters,
            "eps_px2": float(w.eps[0]), "eps_paper": 2e-4, "precision": a.precision,
            "step": f"fot_solve (prep + {a.iters} iterations) + fot_phase",
            "l2": "flushed between steps (256 MB write)",
            "parallelism": f"replicas x{ws} (independent problems)"}


def _max_over_ranks(x, device):
    """The largest of every rank's x (the slowest rank sets the whole job's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _whole_job_value(world_size, n, iters, step_ms):
    """Mpixel*iter/s of the whole job: every rank solves its own n x n problem (weak scaling),
    so the units are world_size * n^2 * iters per step of step_ms (the slowest rank's)."""
    return world_size * n * n * iters / (step_ms * 1e-3) / 1e6


def _workload(n, iters):
    from paper_2512_19072_gb300 import inputs
    w = inputs.config3(n, iters=iters)
    return w


# ----------------------------------------------------------------------------------------
# CPU side: the FP64 oracle, as it stands, on a bounded sample
# ----------------------------------------------------------------------------------------
def _oracle_sample(w, rows, budget_s):
    """Time the oracle's axis pass (its exact FP64 log-sum-exp) on `rows` input rows of the
    workload, repeated until `budget_s` elapsed.  One FOT iteration is 4 passes over n rows,
    so the time of one iteration is (time per row) * 4 n."""
    import torch
    from oracle import fot
    n = w.g.shape[0]
    eps = float(w.eps[0])
    psi = np.full((rows, n), eps * math.log(1.0 / (n * n)))
    t0 = time.perf_counter()
    reps = 0
    while True:
        fot.axis_lse(psi / eps, eps)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    per_row = el / (reps * rows)
    t_iter = per_row * 4 * n
    return {"value": n * n / t_iter / 1e6, "unit": "Mpixel*iter/s", "cores": torch.get_num_threads(),
            "kind": "oracle", "extrapolated": True,
            "sample": f"{reps} x FP64 oracle axis pass over {rows} of {n} rows at n={n} "
                      f"(eps={eps:.4g} px^2); one iteration = 4 n row-passes, scaled"}


def _oracle_full_256(iters):
    """The oracle's whole Algorithm-1 iteration (fot_iterate, FP64) on the 256^2 downsample of
    the single workload, for `iters` iterations: a measured rate, no extrapolation."""
    import torch
    from oracle import fot
    w = _workload(256, iters)
    g = np.asarray(w.g, dtype=np.float32).astype(np.float64)
    G = np.asarray(w.G, dtype=np.float32).astype(np.float64)
    t0 = time.perf_counter()
    fot.fot_iterate(g, G, w.eps, iters)
    el = time.perf_counter() - t0
    return {"workload": w.name, "iters": iters, "seconds": el, "cores": torch.get_num_threads(),
            "value": 256 * 256 * iters / el / 1e6, "unit": "Mpixel*iter/s"}


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = _workload(a.n, a.iters)
    vals = []
    for i in range(a.warmup + a.steps):
        s = _oracle_sample(w, rows=16, budget_s=2.0)
        if i >= a.warmup:
            vals.append(s["value"])
    v = statistics.median(vals)
    s["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpixel*iter/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": a.n * a.n * a.iters / (v * 1e6) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w, a.n, a, ws),
            "cpu_baseline": s,
            "extrapolated": "value: the oracle's FP64 axis pass timed on 16 rows of the 1024^2 "
                            "workload's first iterate and scaled to 4 n row-passes per iteration",
            "oracle_full_solve_256": _oracle_full_256(10),
            "e2e": {"value": v, "unit": "Mpixel*iter/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------
# GPU side
# ----------------------------------------------------------------------------------------
class _Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.rows = []
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ALU rooflines (per SM per clock, times 152 SMs and the maximum SM clock):
#  - MUFU ex2: 32 lanes/clk/SM on sm_103 (GB300 doubles sm_100's special-function rate;
#    ncu's sm__inst_executed_pipe_xu peak agrees), bound of the dense exact pass;
#  - FP32 FFMA: 128 lanes/clk/SM = 256 flop/clk/SM, bound of the banded pass's GEMM loop.
EX2_PER_CLK_PER_SM = 32
FFMA_FLOP_PER_CLK_PER_SM = 256
N_SM = 152


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a kernel, from an ncu
# capture of the current build on the benchmark workload (the capture and its command are in the
# named profiles/ summary).  Keyed by (kernel, n, precision); a kernel that changes since its
# capture must lose its entry (the bench line then reports traffic null).
NCU_TRAFFIC = {
    ("tc_pass_kernel", 1024, "mixed"): {
        "bytes": (4.548096e6 + 0.0 + 8.751104e6 + 5.376e3) / 2,
        "source": "ncu --set full, one row-pass and one column-pass launch (mean), "
                  "profiles/tc_pass_kernel_c3_1024_mixed.md"},
}


def _roofline(n, a, ktimes, work, loop_ms):
    """Roofline of the dominant kernel (largest device time in the event-timed loops): its
    algorithmic work over the CUDA-event time of its own launches, against the unit that
    bounds it.  work = per-step terms by class (banded GEMM, exact window, tensor, dense),
    counted in the timed steps (the event-timed steps repeat them exactly)."""
    peaks, peak_src = _peaks()
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    steps = a.steps
    total_ms = sum(t for t, _ in ktimes.values())
    kernels = {k: {"ms_per_step": t / steps, "launches_per_step": c / steps,
                   "share": t / total_ms if total_ms else None}
               for k, (t, c) in ktimes.items() if c}
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    t_ms, n_launch = ktimes[dom]
    sec = t_ms * 1e-3
    gemm, exact, tensor, dense = (w * steps for w in work)
    dense -= 2.0 * n * n * n * steps            # the phase step's two moment passes (not in the loop)
    ex2_peak = EX2_PER_CLK_PER_SM * N_SM * clk_mhz * 1e6 / 1e12
    ffma_peak = FFMA_FLOP_PER_CLK_PER_SM * N_SM * clk_mhz * 1e6 / 1e12
    if dom == "band_pass_kernel" and gemm >= exact:
        roof = {"bound": "alu", "achieved": 2.0 * gemm / sec / 1e12, "peak": ffma_peak,
                "unit": "TFLOP/s", "work": "2 flop (one FFMA) per window term of the tilted GEMM",
                "peak_source": f"FP32 FFMA {FFMA_FLOP_PER_CLK_PER_SM} flop/clk/SM x {N_SM} SMs x "
                               f"{clk_mhz:.0f} MHz",
                "exact_window_terms": exact / steps}
    elif dom == "band_pass_kernel":
        roof = {"bound": "alu", "achieved": exact / sec / 1e12, "peak": ex2_peak, "unit": "Tex2/s",
                "work": "one exponential per exact-window term",
                "peak_source": f"MUFU ex2 {EX2_PER_CLK_PER_SM}/clk/SM x {N_SM} SMs x {clk_mhz:.0f} MHz",
                "gemm_window_terms": gemm / steps}
    elif dom == "tc_pass_kernel":
        # algorithmic work of the dense separable iteration: 8 n^3 flop per iteration (2 n^3 per
        # axis pass: n rows x n outputs x n terms, one multiply-add each), over the time of the
        # tensor kernel's own launches; the flops it executed (3 BF16 multiply-adds per window
        # term of the union windows) are reported beside it
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        algo = 8.0 * n ** 3 * a.iters * steps
        roof = {"bound": "tensor", "achieved": algo / sec / 1e12, "peak": peak,
                "unit": "TFLOP/s", "work": "8 n^3 flop per iteration (the dense separable contraction of "
                                           "Sec. 3: 4 axis passes of n^3 multiply-adds) over the tensor "
                                           "kernel's event time",
                "peak_source": "cuBLAS bf16 sustained, " + peak_src,
                "executed_tflops": 6.0 * tensor / sec / 1e12,
                "executed_frac": 6.0 * tensor / sec / 1e12 / peak,
                "executed_work": "3 BF16 multiply-adds (split precision) per window term computed",
                "cuda_core_terms_in_kernel": (gemm + exact) / steps}
    elif dom == "axis_pass_kernel":
        roof = {"bound": "alu", "achieved": dense / sec / 1e12, "peak": ex2_peak, "unit": "Tex2/s",
                "work": "one exponential per (row, output, term) of the dense pass",
                "peak_source": f"MUFU ex2 {EX2_PER_CLK_PER_SM}/clk/SM x {N_SM} SMs x {clk_mhz:.0f} MHz"}
    else:                                        # window plan: reads the row, writes the plan
        nbytes = n_launch * (n * n * 4 + n * ((n + 15) // 16) * 12)
        peak = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"bound": "hbm", "achieved": nbytes / sec / 1e9, "peak": peak, "unit": "GB/s",
                "work": "x read once + 3 plan words per (row, tile) written",
                "peak_source": "STREAM copy, " + peak_src}
    tr = NCU_TRAFFIC.get((dom, n, a.precision))
    roof.update({"kernel": dom, "frac": roof["achieved"] / roof["peak"],
                 "traffic": tr["bytes"] if tr else None,
                 "traffic_source": tr["source"] if tr else None,
                 "launches": n_launch, "avg_launch_us": t_ms * 1e3 / max(n_launch, 1),
                 "kernels": kernels, "loop_ms": loop_ms,
                 "dense_equivalent_tflops": 2.0 * 4.0 * a.iters * n ** 3 / (loop_ms * 1e-3) / 1e12,
                 "terms_per_iter": {"band_gemm": work[0] / a.iters, "band_exact": work[1] / a.iters,
                                    "tensor": work[2] / a.iters,
                                    "dense_loop": max(work[3] - 2.0 * n ** 3, 0.0) / a.iters,
                                    "dense_equivalent": 4.0 * n ** 3}})
    return roof


def _timed_steps(step, steps, warmup, flush, stream):
    """Median device time (ms) of `steps` calls of step() after `warmup` untimed ones, with an L2
    flush (a 256 MB write) before every call, outside the events."""
    import torch
    for _ in range(warmup):
        flush.zero_()
        step()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def _sub_single(B, n, prec_name, iters, steps, warmup, flush, stream):
    """The single workload (config 3) at n^2 in one precision: fot_solve + fot_phase per step."""
    import torch
    w = _workload(n, iters)
    g = torch.from_numpy(w.g.astype(np.float32)).cuda()
    G = torch.from_numpy(w.G.astype(np.float32)).cuda()
    prec = {"fp32": B.FOT_FP32, "mixed": B.FOT_MIXED, "bf16": B.FOT_BF16}[prec_name]
    ctx = B.fot_create(n, n, prec)
    phi, Dx, Dy = ctx.empty(), ctx.empty(), ctx.empty()

    def step():
        B.fot_solve(ctx, g, G, w.eps, iters)
        B._check(B._lib.fot_phase(ctx._h, B._ptr(phi), B._ptr(Dx), B._ptr(Dy)), "fot_phase")

    ms = _timed_steps(step, steps, warmup, flush, stream)
    l1, _ = B.fot_marginal_error(ctx)
    ctx.close()
    return {"workload": w.name, "precision": prec_name, "value": n * n * iters / (ms * 1e-3) / 1e6,
            "unit": "Mpixel*iter/s", "ms_per_step": ms, "steps": steps, "marginal_l1": l1}


def _measure_batched(B, prec_name, iters, steps, warmup, stream, with_loop):
    """Config 5 (64 problems of 128^2 .. 512^2) in one precision: one fot_batch_solve per step,
    optionally against a loop of single solves of the same problems."""
    import torch
    from paper_2512_19072_gb300 import inputs
    ws = inputs.config5(iters=iters)
    prec = {"fp32": B.FOT_FP32, "mixed": B.FOT_MIXED}[prec_name]
    gs = [torch.from_numpy(w.g.astype(np.float32)).cuda() for w in ws]
    Gs = [torch.from_numpy(w.G.astype(np.float32)).cuda() for w in ws]
    eps = np.stack([w.eps for w in ws])
    pix_iters = sum(w.g.size for w in ws) * iters
    batch = B.fot_batch_create([w.g.shape for w in ws], prec)
    flush = torch.empty(1, device="cuda")            # the batch's working set is below L2: no flush
    ms_b = _timed_steps(lambda: B.fot_batch_solve(batch, gs, Gs, eps, iters), steps, warmup, flush, stream)
    kernels, tensor = B.fot_batch_info(batch)
    l1 = [B.fot_marginal_error(B.fot_batch_context(batch, q))[0] for q in range(len(ws))]
    out = {"workload": "c5_64_problems_128_to_512", "precision": prec_name, "tensor_path": tensor,
           "value": pix_iters / (ms_b * 1e-3) / 1e6, "unit": "Mpixel*iter/s", "ms_per_step": ms_b,
           "steps": steps, "kernels_per_graph": kernels, "marginal_l1_max": max(l1),
           "marginal_l1_mean": float(np.mean(l1)), "sizes": sorted(int(w.g.shape[0]) for w in ws)}
    if with_loop:
        ctxs = [B.fot_create(*w.g.shape, prec) for w in ws]

        def loop():
            for c, g, G, w in zip(ctxs, gs, Gs, ws):
                B.fot_solve(c, g, G, w.eps, iters)

        ms_l = _timed_steps(loop, max(1, steps // 2), 1, flush, stream)
        out["loop_of_single_solves"] = {"value": pix_iters / (ms_l * 1e-3) / 1e6, "ms": ms_l}
        out["speedup_vs_loop"] = ms_l / ms_b
        for c in ctxs:
            c.close()
    batch.close()
    return out


def _sub_to_tol(B, n, prec_name, tol, max_iters, check_every, flush, stream):
    """Iterations and device time of fot_solve_tol on the single workload until the marginal
    violation sum |Gamma 1 - a| <= tol (Sec. 3), or max_iters."""
    import torch
    w = _workload(n, 1)
    g = torch.from_numpy(w.g.astype(np.float32)).cuda()
    G = torch.from_numpy(w.G.astype(np.float32)).cuda()
    prec = {"fp32": B.FOT_FP32, "mixed": B.FOT_MIXED}[prec_name]
    ctx = B.fot_create(n, n, prec)
    done = [0, 0.0]

    def step():
        done[0], done[1] = B.fot_solve_tol(ctx, g, G, w.eps[:1], max_iters, tol, check_every)

    ms = _timed_steps(step, 1, 1, flush, stream)
    ctx.close()
    return {"precision": prec_name, "tol": tol, "reached": bool(done[1] <= tol), "iters": done[0],
            "violation": done[1], "ms": ms, "max_iters": max_iters, "check_every": check_every}


def run_gpu(a):
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    from paper_2512_19072_gb300 import binding as B

    w = _workload(a.n, a.iters)
    n = a.n
    g = torch.from_numpy(w.g.astype(np.float32)).cuda()
    G = torch.from_numpy(w.G.astype(np.float32)).cuda()
    eps = w.eps
    prec = {"fp32": B.FOT_FP32, "fp32_dense": B.FOT_FP32_DENSE, "mixed": B.FOT_MIXED,
            "bf16": B.FOT_BF16}[a.precision]
    ctx = B.fot_create(n, n, prec)
    phi = ctx.empty()
    Dx = ctx.empty()
    Dy = ctx.empty()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        B.fot_solve(ctx, g, G, eps, a.iters)
        B._check(B._lib.fot_phase(ctx._h, B._ptr(phi), B._ptr(Dx), B._ptr(Dy)), "fot_phase")

    for _ in range(a.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = _Clocks(dev)
    l0 = B.fot_launch_count(ctx)
    split0 = B.fot_work_split(ctx)
    torch.cuda.synchronize()
    evs = []
    loop_ms = []
    passes = 0
    for _ in range(a.steps):
        flush.zero_()                       # L2 flush between steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
        ms_loop, passes = B.fot_loop_time(ctx)
        loop_ms.append(ms_loop)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches = B.fot_launch_count(ctx) - l0
    split1 = B.fot_work_split(ctx)
    work = [(b - a_) / a.steps for a_, b in zip(split0, split1)]   # per step, by class
    clk = clocks.stop()
    # Kernel durations for the roofline: the same steps again with a pair of CUDA events around
    # every kernel of the loop (on the context stream).  The events add about a microsecond per
    # launch, so they stay out of the steps that give `value`; one untimed step creates them.
    B.fot_set_kernel_timing(ctx, True)
    flush.zero_()
    step()
    B.fot_kernel_times(ctx)
    for _ in range(a.steps):
        flush.zero_()
        step()
    ktimes = B.fot_kernel_times(ctx)
    B.fot_set_kernel_timing(ctx, False)
    step_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / a.steps
    if ws > 1:
        step_ms = _max_over_ranks(step_ms, "cuda")
    value = _whole_job_value(ws, n, a.iters, step_ms)

    line = None
    if rank == 0:
        l1, dual = B.fot_marginal_error(ctx)
        loop = statistics.median(loop_ms)
        roof = _roofline(n, a, ktimes, work, loop)
        # end to end through the C ABI with host buffers (H2D of g, G and D2H of phi per step)
        gh = torch.from_numpy(w.g.astype(np.float32)).pin_memory()
        Gh = torch.from_numpy(w.G.astype(np.float32)).pin_memory()
        ph = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        B.fot_solve_phase_host(ctx, gh, Gh, eps, a.iters, phi_host=ph)
        t_e2e = []
        for _ in range(max(2, a.steps // 2)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.fot_solve_phase_host(ctx, gh, Gh, eps, a.iters, phi_host=ph)
            t_e2e.append(time.perf_counter() - t0)
        e2e_v = n * n * a.iters / statistics.median(t_e2e) / 1e6
        cpu = None
        if not a.no_cpu_baseline and ws == 1:
            cpu = _oracle_sample(w, rows=32, budget_s=12.0)
        # the plain FP32 form on the same workload and steps (the metric compares the two)
        compare = None
        if a.precision == "mixed" and not a.no_compare:
            c32 = B.fot_create(n, n, B.FOT_FP32)

            def step32():
                B.fot_solve(c32, g, G, eps, a.iters)
                B._check(B._lib.fot_phase(c32._h, B._ptr(phi), B._ptr(Dx), B._ptr(Dy)), "fot_phase")

            for _ in range(a.warmup):
                flush.zero_()
                step32()
            ms32 = []
            for _ in range(a.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step32()
                e1.record(stream)
                e1.synchronize()
                ms32.append(e0.elapsed_time(e1))
            l1_32, _ = B.fot_marginal_error(c32)
            v32 = n * n * a.iters / (statistics.mean(ms32) * 1e-3) / 1e6
            compare = {"precision": "fp32", "value": v32, "ms_per_step": statistics.mean(ms32),
                       "marginal_l1": l1_32, "marginal_l1_diff": abs(l1 - l1_32),
                       "mixed_speedup": value / v32}
            c32.close()
        sub = None
        if not a.no_sub and ws == 1 and n == 1024:
            sub = {"note": "the same library on other workloads, each timed as the main line "
                           "(L2 flush between steps, CUDA events); not part of value"}
            sub["c3_2048"] = [_sub_single(B, 2048, p_, a.iters, 3, 2, flush, stream) for p_ in ("mixed", "fp32")]
            sub["c3_1024_single_bf16"] = _sub_single(B, 1024, "bf16", a.iters, 3, 2, flush, stream)
            sub["c3_1024_single_bf16"]["error_bound"] = "2^-6 eps per half-step (split-BF16 mixed: 2^-15 eps)"
            sub["c5_batched"] = [_measure_batched(B, p_, 200, 3, 1, stream, with_loop=(p_ == "mixed"))
                                 for p_ in ("mixed", "fp32")]
            sub["c3_1024_to_violation_1e-4"] = [_sub_to_tol(B, n, p_, 1e-4, 4000, 100, flush, stream)
                                                 for p_ in ("mixed", "fp32")]
        line = {"metric": METRIC if n == 1024 else METRIC.replace("1024^2", f"{n}^2"), "value": value, "unit": "Mpixel*iter/s", "n_gpus": ws,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": step_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"mixed": "bf16+f32", "bf16": "bf16x1+f32"}.get(a.precision, "f32"),
                "data": "synthetic (seeded two-Gaussian beam -> 12-shape composite target)",
                "config": _config(w, n, a, ws),
                "marginal_l1": l1, "dual_objective": dual,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_v, "unit": "Mpixel*iter/s",
                        "h2d_bytes_per_step": 2 * n * n * 4, "d2h_bytes_per_step": n * n * 4},
                "gpu_launches": launches, "clocks": clk, "fp32_form": compare, "sub_records": sub,
                "paper_context": "1024^2, 200 iterations: 76 s Core i7 (2.76 Mpixel*iter/s), "
                                 "8.5 s T4 (24.7 Mpixel*iter/s)"}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_batched(a):
    """64 problems, n_i in {128,...,512}, eps 32 -> 1 px^2 over 200 iterations: one batched
    solve (multi-problem launches replayed as a CUDA graph) vs a loop of single solves."""
    import torch
    from paper_2512_19072_gb300 import binding as B
    from paper_2512_19072_gb300 import inputs
    ws = _workload_batched = inputs.config5(iters=a.iters)
    prec = {"fp32": B.FOT_FP32, "fp32_dense": B.FOT_FP32, "mixed": B.FOT_MIXED}[a.precision]
    gs = [torch.from_numpy(w.g.astype(np.float32)).cuda() for w in ws]
    Gs = [torch.from_numpy(w.G.astype(np.float32)).cuda() for w in ws]
    eps = np.stack([w.eps for w in ws])
    pix_iters = sum(w.g.size for w in ws) * a.iters
    batch = B.fot_batch_create([w.g.shape for w in ws], prec)
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        B.fot_batch_solve(batch, gs, Gs, eps, a.iters)
    torch.cuda.synchronize()
    clocks = _Clocks(torch.cuda.current_device())
    t_b = []
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.fot_batch_solve(batch, gs, Gs, eps, a.iters)
        e1.record(stream)
        t_b.append((e0, e1))
    torch.cuda.synchronize()
    ms_b = statistics.median(e0.elapsed_time(e1) for e0, e1 in t_b)
    kernels, tensor = B.fot_batch_info(batch)
    ctxs = [B.fot_create(*w.g.shape, prec) for w in ws]
    def loop():
        for c, g, G, w in zip(ctxs, gs, Gs, ws):
            B.fot_solve(c, g, G, w.eps, a.iters)
    loop()
    torch.cuda.synchronize()
    t_l = []
    for _ in range(max(1, a.steps // 2)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loop()
        e1.record(stream)
        t_l.append((e0, e1))
    torch.cuda.synchronize()
    ms_l = statistics.median(e0.elapsed_time(e1) for e0, e1 in t_l)
    clk = clocks.stop()
    l1 = [B.fot_marginal_error(B.fot_batch_context(batch, q))[0] for q in range(len(ws))]
    line = {"metric": "FOT Mpixel*iter/s, 64-problem uneven batch (config 5)",
            "value": pix_iters / (ms_b * 1e-3) / 1e6, "unit": "Mpixel*iter/s", "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_b, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32" if tensor else "f32",
            "data": "synthetic (seeded Gaussian / two-Gaussian beams -> 2-6 shape targets)",
            "config": {"workload": "c5_64_problems_128_to_512", "iters_per_solve": a.iters,
                       "eps": "geometric 32 -> 1 px^2", "precision": a.precision,
                       "sizes": sorted(int(w.g.shape[0]) for w in ws),
                       "step": "fot_batch_solve (one CUDA graph launch)"},
            "loop_of_single_solves": {"value": pix_iters / (ms_l * 1e-3) / 1e6, "ms": ms_l},
            "speedup_vs_loop": ms_l / ms_b, "kernels_per_graph": kernels, "tensor_path": tensor,
            "marginal_l1_max": max(l1), "clocks": clk}
    print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    batch.close()
    return 0


def run_stopping(a):
    """The single workload with the convergence stop: fot_solve_tol (at most --iters
    iterations, a violation check every --check-every) + fot_phase per step, against
    fot_solve with the same number of iterations (the cost of the checks)."""
    import torch
    from paper_2512_19072_gb300 import binding as B
    w = _workload(a.n, a.iters)
    n = a.n
    g = torch.from_numpy(w.g.astype(np.float32)).cuda()
    G = torch.from_numpy(w.G.astype(np.float32)).cuda()
    prec = {"fp32": B.FOT_FP32, "fp32_dense": B.FOT_FP32_DENSE, "mixed": B.FOT_MIXED}[a.precision]
    ctx = B.fot_create(n, n, prec)
    phi, Dx, Dy = ctx.empty(), ctx.empty(), ctx.empty()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    done = [0, 0.0]

    def step_tol():
        done[0], done[1] = B.fot_solve_tol(ctx, g, G, w.eps, a.iters, a.tol, a.check_every)
        B._check(B._lib.fot_phase(ctx._h, B._ptr(phi), B._ptr(Dx), B._ptr(Dy)), "fot_phase")

    def step_fixed():
        B.fot_solve(ctx, g, G, w.eps[:done[0]], done[0])   # one eps per iteration
        B._check(B._lib.fot_phase(ctx._h, B._ptr(phi), B._ptr(Dx), B._ptr(Dy)), "fot_phase")

    def timed(step):
        for _ in range(a.warmup):
            flush.zero_()
            step()
        ms = []
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    clocks = _Clocks(torch.cuda.current_device())
    ms_tol = timed(step_tol)
    clk = clocks.stop()
    iters, tv = done
    ms_fixed = timed(step_fixed)
    cfg = _config(w, n, a, 1)
    cfg.update({"step": "fot_solve_tol (prep + at most %d iterations, a check every %d) + fot_phase"
                        % (a.iters, a.check_every), "tol": a.tol, "check_every": a.check_every,
                "iters_done": iters})
    line = {"metric": "FOT Mpixel*iter/s to a marginal-violation tolerance", "value": n * n * iters / (ms_tol * 1e-3) / 1e6,
            "unit": "Mpixel*iter/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms_tol, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32" if a.precision == "mixed" else "f32", "data": "synthetic",
            "config": cfg, "violation": tv, "fixed_iters_ms_per_step": ms_fixed,
            "check_overhead": ms_tol / ms_fixed - 1.0, "clocks": clk}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_intensity(a):
    """The L1 intensity loss (Sec. 5) of the single workload's phase after one solve: each
    step is one fot_intensity_loss call (two FFT passes and two reductions), timed with CUDA
    events, L2 flushed between steps.  Algorithmic traffic 44 n^2 bytes per call: the row
    pass reads log a and phi and writes the spectrum (8 + 8), the column pass reads it and
    writes I (8 + 4), the reductions read I, read log b and I and rewrite I (4 + 12)."""
    import torch
    from paper_2512_19072_gb300 import binding as B
    w = _workload(a.n, a.iters)
    n = a.n
    g = torch.from_numpy(w.g.astype(np.float32)).cuda()
    G = torch.from_numpy(w.G.astype(np.float32)).cuda()
    ctx = B.fot_create(n, n, B.FOT_MIXED)
    B.fot_solve(ctx, g, G, w.eps, a.iters)
    phi, _, _ = B.fot_phase(ctx)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        loss = B.fot_intensity_loss(ctx, phi)
    ms = []
    for _ in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loss = B.fot_intensity_loss(ctx, phi)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    nbytes = 44.0 * n * n
    peaks, peak_src = _peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    line = {"metric": "FOT L1 intensity loss evaluations/s", "value": 1e3 / t, "unit": "evaluations/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": w.name, "n": n, "phase_from": f"fot_solve ({a.iters} iterations, mixed) + fot_phase",
                                            "l2": "flushed between steps (256 MB write)"},
            "loss": loss,
            "roofline": {"bound": "hbm", "achieved": nbytes / (t * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": nbytes / (t * 1e-3) / 1e9 / peak, "traffic": None,
                         "work": "44 n^2 bytes per evaluation", "peak_source": "STREAM copy, " + peak_src}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_sweep(a):
    """Fig. 3 of Sec. 5: the L1 intensity loss |F[g e^{2 pi i phi}]|^2 - G^2 of the phase after
    T iterations, against eps (paper units), for FOT (this build's mixed form) and cFOT (FP32
    exponential domain), on the two-Gaussian beam -> 12-shape target at n^2 (512 by default for
    this workload).  One solve per (form, eps) continued with fot_resume between the iteration
    counts (fixed eps, so the same iterates as separate solves); cFOT restarts for each count.
    A cFOT run whose potentials leave the FP32 range is reported as unstable."""
    import torch
    from paper_2512_19072_gb300 import binding as B
    n = a.n if a.n != 1024 else 512
    w = _workload(n, 1)
    g = torch.from_numpy(w.g.astype(np.float32)).cuda()
    G = torch.from_numpy(w.G.astype(np.float32)).cuda()
    eps_list = [5e-5, 1e-4, 2e-4, 5e-4, 1e-3, 2e-3, 5e-3, 1e-2, 2e-2, 5e-2, 1e-1]
    iter_list = [50, 100, 200, 400]
    table = {"fot": {}, "cfot": {}}
    ctx = B.fot_create(n, n, B.FOT_MIXED)
    t0 = time.perf_counter()
    for e in eps_list:
        row, done = [], 0
        for T in iter_list:
            if done == 0:
                B.fot_solve(ctx, g, G, [e], T, eps_units=B.FOT_EPS_PAPER)
            else:
                B.fot_resume(ctx, [e], T - done, eps_units=B.FOT_EPS_PAPER)
            done = T
            phi, _, _ = B.fot_phase(ctx)
            row.append(B.fot_intensity_loss(ctx, phi))
        table["fot"][f"{e:g}"] = row
        crow = []
        for T in iter_list:
            try:
                B.fot_cfot_solve(ctx, g, G, [e], T, eps_units=B.FOT_EPS_PAPER)
                phi, _, _ = B.fot_phase(ctx)
                crow.append(B.fot_intensity_loss(ctx, phi))
            except B.FotError as err:
                crow.append("unstable" if B.STATUS.get(err.status) == "FOT_ENONFINITE" else str(err))
        table["cfot"][f"{e:g}"] = crow
    el = time.perf_counter() - t0
    ctx.close()
    line = {"metric": "L1 intensity loss vs eps and iterations (Fig. 3)", "value": None, "unit": "L1",
            "n_gpus": 1, "higher_is_better": False, "dtype": "bf16+f32 (FOT), f32 (cFOT)",
            "data": "synthetic (seeded two-Gaussian beam -> 12-shape composite target)",
            "config": {"workload": w.name, "n": n, "eps_paper": eps_list, "iterations": iter_list,
                       "eps_px2": [e * n * n for e in eps_list]},
            "loss": table, "seconds": el}
    print(json.dumps(line), flush=True)
    return 0


def run_cfot(a):
    """cFOT (FFT convolutions, exponential domain, FP32) against FOT (banded passes, the
    context's mixed form) per iteration, on two beams over a flat floor at n^2 and a large
    eps (cFOT fails at the benchmark workload's eps: its u, V leave the FP32 range).  Each step
    is one solve of --iters iterations, L2 flushed between steps."""
    import torch
    from paper_2512_19072_gb300 import binding as B
    n = a.n
    j = np.arange(n)[:, None]
    k = np.arange(n)[None, :]
    g = torch.from_numpy((np.exp(-((j - 0.45 * n) ** 2 + (k - 0.55 * n) ** 2) / (2 * (n / 5) ** 2)) + 1.0)
                         .astype(np.float32)).cuda()
    G = torch.from_numpy((np.exp(-((j - 0.55 * n) ** 2 + (k - 0.40 * n) ** 2) / (2 * (n / 4) ** 2)) + 1.0)
                         .astype(np.float32)).cuda()
    ctx = B.fot_create(n, n, B.FOT_MIXED)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(a.warmup):
            fn()
        B.fot_sync(ctx)
        ms = []
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        B.fot_sync(ctx)
        return statistics.median(ms)

    failed = None
    try:
        t_c = timed(lambda: B.fot_cfot_solve(ctx, g, G, a.cfot_eps, a.iters))
        l1_c, _ = B.fot_marginal_error(ctx)
        _, psi_c = B.fot_potentials(ctx)
    except B.FotError as e:                  # the exponential-domain iteration left FP32
        failed, t_c, l1_c, psi_c = str(e), float("nan"), None, None
    t_f = timed(lambda: B.fot_solve(ctx, g, G, a.cfot_eps, a.iters))
    l1_f, _ = B.fot_marginal_error(ctx)
    _, psi_f = B.fot_potentials(ctx)
    diff = None
    if psi_c is not None:
        fin = torch.isfinite(psi_f)
        diff = float((psi_c[fin] - psi_f[fin]).abs().max() / psi_f[fin].abs().max())
    line = {"metric": "cFOT Mpixel*iter/s (FFT convolutions) vs FOT", "value": n * n * a.iters / (t_c * 1e-3) / 1e6,
            "unit": "Mpixel*iter/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_c,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "two beams over a flat floor", "n": n, "iters_per_solve": a.iters,
                       "eps_px2": a.cfot_eps, "l2": "flushed between steps (256 MB write)"},
            "cfot_ms_per_iter": t_c / a.iters, "fot_mixed_ms_per_iter": t_f / a.iters,
            "marginal_l1": {"cfot": l1_c, "fot": l1_f}, "psi_rel_diff": diff, "cfot_failed": failed}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batched":
        return run_batched(a)
    if a.workload == "stopping":
        return run_stopping(a)
    if a.workload == "intensity":
        return run_intensity(a)
    if a.workload == "cfot":
        return run_cfot(a)
    if a.workload == "sweep":
        return run_sweep(a)
    return run_gpu(a)


if __name__ == "__main__":
    sys.exit(main())
