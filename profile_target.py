"""Profiling target: plans one synthetic workload and runs the solver for a
fixed number of Newton iterations (a representative mix of every kernel of
the hot path), for use under ncu:

    python profile_target.py --config c2 --precision fp32 --newton 3
    python profile_target.py --config c2 --precision tc --newton 2 \
        --warm-newton 60      # late-phase CG iterations inside the NVTX range "profiled"
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "c3s", "f2"],
                    help="c3: the megascale geometry (M = D = 1e6, N = 100, lambda linear in "
                         "[0, 9e5], band +-10 sqrt(lambda); products only, timed with CUDA events); "
                         "c3s: the same geometry at 1/8 size (M = D = 131072, N = 100, "
                         "lambda linear in [0, 0.9 M], band +-10 sqrt(lambda); products only); "
                         "f2: the loop detector at the paper's size (M = 1210581, N = 151, "
                         "D = 1076, lambda_d = d^2, gamma 1e-5)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed", "tc"])
    ap.add_argument("--newton", type=int, default=3)
    ap.add_argument("--op", default="fit", choices=["fit", "hvp", "fwd", "adj"],
                    help="fit: the solver; hvp/fwd/adj: --reps single products")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warm-newton", type=int, default=0,
                    help="fit: first run this many Newton iterations unprofiled, then continue "
                         "(stage 2) from there inside the NVTX range 'profiled' (late-phase CG)")
    args = ap.parse_args()

    import torch

    import paper_2404_02844_gb300 as tomo
    import workloads
    from paper_2404_02844_gb300 import build

    build.build()
    if args.config in ("c3", "c3s"):
        M = D = 1_000_000 if args.config == "c3" else 131072
        N = 100
        lam = workloads.probe_intensities(D, 0.9 * M)
        with tomo.Plan(M, N, lam, 10.0, 1e-3, precision=args.precision) as pl:
            g = torch.Generator(device="cuda").manual_seed(1)
            X = torch.rand(M, N, dtype=torch.float64, device="cuda", generator=g)
            pl.hvp(X)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for _ in range(args.reps):
                pl.hvp(X)
            ev1.record()
            torch.cuda.synchronize()
            print(f"{args.config} {args.precision}: {args.reps} x hvp, {ev0.elapsed_time(ev1) / args.reps:.3f} ms each")
        return
    w = {"c1": workloads.config_c1, "c2": workloads.config_c2,
         "f2": lambda: workloads.config_f2(M=1210581, D=1076, gamma=1e-5)}[args.config]()
    P = torch.from_numpy(w.P).cuda()
    with tomo.Plan.from_workload(w, precision=args.precision) as pl:
        if args.op != "fit":
            g = torch.Generator(device="cuda").manual_seed(1)
            X = torch.rand(w.M, w.N, dtype=torch.float64, device="cuda", generator=g)
            Y = torch.rand(w.D, w.N, dtype=torch.float64, device="cuda", generator=g)
            fn = {"hvp": lambda: pl.hvp(X), "fwd": lambda: pl.apply_F(X),
                  "adj": lambda: pl.apply_Ft(Y)}[args.op]
            t0 = time.perf_counter()
            for _ in range(args.reps):
                fn()
            torch.cuda.synchronize()
            print(f"{w.name} {args.precision}: {args.reps} x {args.op}, "
                  f"{(time.perf_counter() - t0) / args.reps * 1e3:.3f} ms each")
            return
        if args.warm_newton > 0:
            Th0, _ = pl.fit(P, max_newton=args.warm_newton, eps_kkt=0.0)
            # one unprofiled continuation (graph capture), then the profiled one
            pl.fit(P, Th0.clone(), max_newton=args.newton, eps_kkt=0.0, start_stage=2)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("profiled")
            t0 = time.perf_counter()
            _, rep = pl.fit(P, Th0.clone(), max_newton=args.newton, eps_kkt=0.0, start_stage=2)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            torch.cuda.nvtx.range_pop()
        else:
            t0 = time.perf_counter()
            _, rep = pl.fit(P, max_newton=args.newton, eps_kkt=0.0)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
    print(f"{w.name} {args.precision}: {args.newton} Newton iterations, "
          f"{rep['cg_total']} CG products, {rep['ls_total']} line-search trials, "
          f"{rep['kernels']} kernels, {dt:.3f}s, f={rep['f']:.12e}")


if __name__ == "__main__":
    main()
