"""Benchmark: time-to-tolerance (relative objective gap 1e-8) and
POVM-elem*iters/s of the detector-tomography solver on the synthetic
M=4096, N=128, D=8192 workload (127-bin detector, efficiency 0.8, dark counts
1e-4/bin, lambda linear in [0, 3000], 1e7 shots, gamma 1e-2, band
+-10 sqrt(lambda)), chosen form against the plain FP64 GPU solver.

A step is one full two-stage solve (Algorithm 3) from Theta^(0) = 1/N until the
objective is within 1e-8 (relative) of the optimum certified by the FP64
oracle (tests/golden/fstar_c2.json, written by tests/golden/make_fstar.py);
the gap of every result is checked afterwards with a double-precision
objective, outside the timing.  The chosen form runs the CG Hessian products
on the tensor cores (tcgen05, bf16 hi/lo split, f32 accumulation) with float
CG vectors, the gradient and line-search products as FP32 SIMT contractions,
and keeps Theta, the residual (refreshed by an FP64 product every 8 Newton
iterations) and the reductions in FP64.  The plain FP64 GPU solver and the
FP32 form are each timed to the same tolerance beside it.  Prints one JSON
line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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

import workloads  # noqa: E402

METRIC = "time-to-tolerance (rel. obj gap 1e-8) and POVM-elem·iters/s, chosen vs plain"
UNIT = "POVM-elem*iters/s"
GAP = 1e-8
CHOSEN = "tc"
# DRAM bytes (read + write) of one tensor-core Hessian product (forward and
# adjoint contraction and their finish kernels) from one `ncu` capture of the
# late-phase CG on this workload (cold caches), or None when the kernels have
# changed since the counters were taken.
TC_HVP_DRAM_BYTES = None
WORKLOAD = "c2: M=4096 N=128 D=8192, 127-bin eta=0.8 dark=1e-4, lambda lin [0,3000], 1e7 shots, gamma=1e-2, band +-10sqrt(lambda)"


def load_fstar():
    with open(os.path.join(ROOT, "tests", "golden", "fstar_c2.json")) as fh:
        return json.load(fh)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("TOMO_BENCH_BACKEND") != "gloo" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- oracle
def oracle_per_op(w, reps: int = 3):
    """The FP64 CPU oracle as it stands, on the host cores: mean time of each
    operation of the solve (Table ops) on the workload, in ms."""
    import oracle
    pr = oracle.Problem.from_workload(w)
    rng = np.random.default_rng(1)
    Th = workloads.random_feasible_theta(w.M, w.N, rng)
    V = rng.standard_normal((w.M, w.N))
    ops = {"hvp": lambda: pr.hvp(V), "objective": lambda: pr.objective(w.P, Th),
           "gradient": lambda: pr.gradient(w.P, Th), "projection": lambda: pr.project_rows(V)}
    out = {}
    for name, fn in ops.items():
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        out[name] = 1e3 * (time.perf_counter() - t0) / reps
    return out, oracle.num_threads()


def oracle_projection(per_op, counts):
    """Time to tolerance of the oracle's own solve, from its per-operation
    times and its own operation counts to the tolerance (one Hessian product
    per CG step, one objective per line-search trial, one gradient and one
    projection per Newton iteration)."""
    it = counts["iters_s1"] + counts["iters_s2"]
    ms = (counts["cg_total"] * per_op["hvp"] + counts["ls_total"] * per_op["objective"]
          + it * (per_op["gradient"] + per_op["projection"]))
    return ms / 1e3, it


def run_reference(args, world, rank):
    """The FP64 CPU oracle as it stands, on the host cores.  Each step times
    one of each of its operations on the workload (a bounded sample); the
    line's value scales those times by the oracle's own operation counts to
    the tolerance (its full solve from Theta = 1/N to the certified gap,
    recorded by tests/golden/make_fstar.py --theta-tol), giving its
    POVM-elem*iters/s over that solve."""
    if rank != 0:
        return
    w = workloads.config_c2()
    gold = load_fstar()
    counts = gold.get("theta_tol_run")
    if counts is None:
        run_reference_sample(args, w)
        return
    for _ in range(args.warmup):
        oracle_per_op(w, reps=1)
    per_steps, t_tot = [], 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        per, cores = oracle_per_op(w, reps=1)
        t_tot += time.perf_counter() - t0
        per_steps.append(per)
    per = {k: statistics.median(p[k] for p in per_steps) for k in per_steps[0]}
    ttt, it = oracle_projection(per, counts)
    value = w.M * w.N * it / ttt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": 1, "seq_len": w.M,
                   "parallelism": "host cores (OpenMP)", "l2": "n/a (CPU)"},
        "time_to_tolerance_s": ttt,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": (f"per step one Hessian product, objective, gradient and row "
                                    f"projection of the FP64 C oracle on c2 (median over steps), "
                                    f"scaled by the oracle's own counts to the tolerance "
                                    f"({it} Newton iterations, {counts['cg_total']} Hessian "
                                    f"products, {counts['ls_total']} line-search objectives)"),
                         "per_op_ms": per},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_sample(args, w, iters: int = 4):
    """Reference arm without the oracle's counts to the tolerance: each step
    times the oracle's first `iters` Newton iterations of the same solve."""
    import oracle
    pr = oracle.Problem.from_workload(w)
    for _ in range(min(args.warmup, 1)):
        pr.fit(w.P, max_newton=1, eps_kkt=0.0)
    times, n_it = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, rep, _ = pr.fit(w.P, max_newton=iters, eps_kkt=0.0)
        times.append(time.perf_counter() - t0)
        n_it += rep["iters_s1"] + rep["iters_s2"]
    T = sum(times)
    value = w.M * w.N * n_it / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": 1, "seq_len": w.M,
                   "parallelism": "host cores (OpenMP)", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"first {iters} Newton iterations of the c2 solve per step (FP64 C oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chosen", choices=["chosen", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 and FP32 legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--plain-limit-s", type=float, default=900.0,
                    help="wall-clock bound of the plain FP64 solve")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    import paper_2404_02844_gb300 as tomo
    from paper_2404_02844_gb300 import build as tomo_build

    tomo_build.build()
    torch.cuda.set_device(local)
    gold = load_fstar()
    f_star = gold["f_star"]
    f_star_status = gold.get("status", "certified")
    f_target = f_star * (1.0 + 0.5 * GAP)

    w = workloads.config_c2()
    M, N, D = w.M, w.N, w.D
    P = torch.from_numpy(w.P).cuda()
    l2_flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def flush():
        l2_flush.fill_(1.0)

    def timed(fn):
        flush()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    chosen = tomo.Plan.from_workload(w, precision=CHOSEN)
    lo, hi = chosen.bands()
    nnz = int(np.sum(np.maximum(hi - lo + 1, 0)))

    for k in range(args.warmup):
        # the last warm-up also captures the CUDA graphs of the profiled solve
        chosen.fit(P, f_target=f_target, profile=1 if k == args.warmup - 1 else 0)
    torch.cuda.synchronize()

    # ---- timed region: K full solves, L2 flushed before each -------------
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times, iters, reps = [], [], []
    launches0 = tomo.tomo_kernel_launches()
    for k in range(args.steps):
        barrier(world)
        # the last timed solve also records CUDA events around every Hessian
        # product (the roofline's live duration); the others record none
        (Th, rep), t = timed(lambda: chosen.fit(P, f_target=f_target,
                                               profile=1 if k == args.steps - 1 else 0))
        times.append(t)
        iters.append(rep["iters_s1"] + rep["iters_s2"])
        reps.append(rep)
    launches = tomo.tomo_kernel_launches() - launches0
    clk = clocks.stop()
    barrier(world)
    T = max_over_ranks(world, sum(times))
    # tolerance check (excluded from the timing): FP64 objective of the result
    f_final = chosen.objective(P, Th)
    gap = (f_final - f_star) / f_star
    units = M * N * sum(iters) * world
    value = units / T
    ttt = T / args.steps

    # dominant kernel: the CG Hessian product (forward + adjoint band
    # contraction on the tensor cores and their finish kernels), timed live
    # with CUDA events on the plan stream inside the last timed solve
    hvp_ms = sum(r["fwd_ms"] + r["adj_ms"] for r in reps) / max(1, sum(r["fwd_count"] for r in reps))
    flops = 4.0 * nnz * N           # 2 F^T (F v): two band contractions of 2 nnz N flop
    peaks = measured_peaks()
    # the product runs inside a seconds-long solve: sustained bf16 peak
    peak = peaks.get("bf16_tflops_sustained")
    peak_src = "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, seconds-long loop)"
    if peak is None:
        peak, peak_src = 1700.0, "fallback 1.7 PFLOP/s sustained bf16 (profiling recipe)"
    achieved = flops / (hvp_ms * 1e-3) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": TC_HVP_DRAM_BYTES,
                "traffic_unit": "bytes per Hessian product (ncu dram read+write, cold caches; contractions + finish kernels)",
                "kernel": "CG Hessian product: k_transpose_split + k_band_tc<fwd> + k_tc_finish<fwd> + k_band_tc<adj> + k_tc_finish<adj>",
                "avg_launch_ms": hvp_ms, "algorithmic_flops_per_launch": flops,
                "peak_source": peak_src,
                # the bf16 hi/lo split issues 3 MMAs per slice: issued tensor work
                "tensor_issue_frac": 3.0 * achieved / peak}

    # ---- end to end through the C ABI with host buffers (one solve) --------
    P_host = torch.from_numpy(w.P).pin_memory().numpy()
    Th_host = torch.empty((M, N), dtype=torch.float64).pin_memory().numpy()
    flush()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rep_e = chosen.fit(P_host, Th_host, f_target=f_target, warm_start=0)
    e2e_t = time.perf_counter() - t0
    f_e2e = chosen.objective(P_host, Th_host)
    iters_e = rep_e["iters_s1"] + rep_e["iters_s2"]
    e2e_T = max_over_ranks(world, e2e_t)
    e2e_value = M * N * iters_e * world / e2e_T

    # ---- GPU per-operation times (same operations as the oracle's) --------
    def op_ms(fn, reps_=20):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps_):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps_

    rng = np.random.default_rng(1)
    Th_r = torch.from_numpy(workloads.random_feasible_theta(M, N, rng)).cuda()
    V_r = torch.from_numpy(rng.standard_normal((M, N))).cuda()
    gpu_ops = {"hvp_tc": op_ms(lambda: chosen.hvp(V_r)),
               "objective_fp64": op_ms(lambda: chosen.objective(P, Th_r)),
               "objective_and_gradient_fp32": op_ms(lambda: chosen.objective(P, Th_r, want_grad=True)),
               "projection": op_ms(lambda: chosen.project_simplex(V_r))}

    # ---- plain FP64 and FP32 GPU solvers, same workload and tolerance ------
    forms = {}
    if not args.no_plain:
        for prec, limit in (("fp64", args.plain_limit_s), ("fp32", 300.0)):
            with tomo.Plan.from_workload(w, precision=prec) as pl:
                pl.fit(P, max_newton=3)          # graphs captured outside the timing
                gpu_ops[f"hvp_{prec}"] = op_ms(lambda: pl.hvp(V_r), 5)
                (Thp, repp), tp = timed(lambda: pl.fit(P, f_target=f_target, max_newton=100000,
                                                       max_seconds=limit))
                fp = pl.objective(P, Thp)
            itp = repp["iters_s1"] + repp["iters_s2"]
            forms[prec] = {"time_to_tolerance_s": tp, "value": M * N * itp / tp, "unit": UNIT,
                           "newton_iters": [repp["iters_s1"], repp["iters_s2"]],
                           "cg_total": repp["cg_total"], "ls_total": repp["ls_total"],
                           "rel_gap": (fp - f_star) / f_star, "stop": repp["stop_name"],
                           "chosen_speedup": tp / ttt}

    # ---- CPU baseline: the oracle's per-operation times ---------------------
    cpu = None
    if rank == 0 and not args.no_cpu:
        per, cores = oracle_per_op(w)
        counts = gold.get("theta_tol_run")
        cpu = {"unit": UNIT, "cores": cores, "kind": "oracle", "per_op_ms": per}
        if counts:
            t_or, it_or = oracle_projection(per, counts)
            cpu.update({"value": M * N * it_or / t_or, "time_to_tolerance_s": t_or,
                        "sample": (f"one Hessian product, objective, gradient and row projection "
                                   f"of the FP64 C oracle on c2 (3 calls each, all host cores), "
                                   f"scaled by the oracle's own counts to the tolerance ({it_or} "
                                   f"Newton iterations, {counts['cg_total']} Hessian products, "
                                   f"{counts['ls_total']} line-search objectives)")})
        else:
            cpu.update({"value": M * N * 1e3 / per["hvp"], "unit": "POVM-elem*HVPs/s",
                        "sample": "one Hessian product of the FP64 C oracle on c2 (3 calls)"})

    if rank == 0:
        plain = forms.get("fp64")
        line = {
            "metric": METRIC,
            "time_to_tolerance_s": ttt,
            "chosen_speedup_vs_plain_fp64": plain["chosen_speedup"] if plain else None,
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * ttt, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3/f32/f64",
            "data": "synthetic (seeded PCG64; stands in for the paper's experimental data)",
            "config": {"workload": WORKLOAD, "global_batch": world, "seq_len": M,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "form": "chosen: tensor-core CG Hessian products (bf16 hi/lo x3) with float CG vectors, FP32 line-search products and gradient, FP64 Theta/residual refresh/objective/reductions",
                       "l2": "flushed (512 MB write) before every timed solve"},
            "rel_gap": gap,
            "f_star": f_star,
            "f_star_status": f_star_status,
            "newton_iters": iters,
            "cg_total": [r["cg_total"] for r in reps],
            # companion rate: POVM elements times CG Hessian products per second
            "hvp_rate": {"value": M * N * sum(r["cg_total"] for r in reps) * world / T,
                         "unit": "POVM-elem*HVPs/s"},
            "stop": reps[-1]["stop_name"],
            "plain_fp64": plain,
            "fp32": forms.get("fp32"),
            "gpu_per_op_ms": gpu_ops,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": D * N * 8,
                    "d2h_bytes_per_step": M * N * 8,
                    "time_to_tolerance_s": e2e_T, "rel_gap": (f_e2e - f_star) / f_star,
                    "steps": 1},
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    chosen.close()


if __name__ == "__main__":
    main()
