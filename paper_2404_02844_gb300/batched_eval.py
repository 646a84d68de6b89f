"""Throughput of batched solves on the c4 population (independent instances,
M ~ U{256..max_M}, N ~ U{8..128}, D = 2M, each at gamma in
{1e-4, 1e-3, 1e-2, 1e-1}) through tomo_fit_batched:

    python -m paper_2404_02844_gb300.batched_eval [--instances 8] [--max-m 1024]
        [--precision fp32] [--concurrency 8] [--eps-kkt 1e-6] [--max-newton 200]

Solves every (instance, gamma) pair one at a time (concurrency 1, default
schedules) and with the worker pool (with and without the plan-time
autotuner), and prints one JSON line: solves per second, Newton iterations
and the agreement of the objectives between the runs.  The tolerance and the
iteration cap bound the work: the small-gamma instances are ill-conditioned.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=8)
    ap.add_argument("--max-m", type=int, default=1024)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tc", "mixed", "fp64"])
    ap.add_argument("--concurrency", type=int, default=8)
    ap.add_argument("--eps-kkt", type=float, default=1e-6)
    ap.add_argument("--max-newton", type=int, default=200)
    ap.add_argument("--serial-sample", type=int, default=0,
                    help="> 0: time one-at-a-time solves on the first K problems only "
                         "(the full serial pass is skipped)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--fit-seconds", type=float, default=0.0,
                    help="> 0: wall-clock bound of every solve")
    ap.add_argument("--data-workers", type=int, default=1,
                    help="host processes that generate the instances (spawned before any GPU call)")
    args = ap.parse_args()

    import torch

    import paper_2404_02844_gb300 as tomo
    import workloads as W
    from paper_2404_02844_gb300 import build

    build.build()
    t0 = time.perf_counter()
    if args.data_workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(args.data_workers, mp_context=mp.get_context("spawn")) as ex:
            inst = list(ex.map(W.config_c4_instance, range(args.instances),
                               [args.max_m] * args.instances))
    else:
        inst = W.config_c4(n_instances=args.instances, max_M=args.max_m)
    t_data = time.perf_counter() - t0
    print(json.dumps({"data_s": t_data}), flush=True)
    lim = dict(max_seconds=args.fit_seconds) if args.fit_seconds > 0 else {}
    problems = [(w, g) for w in inst for g in W.C4_GAMMAS]
    Ps = [torch.from_numpy(w.P).cuda() for w, _ in problems]

    def run(conc, autotune):
        Ths = [torch.empty(w.M, w.N, dtype=torch.float64, device="cuda") for w, _ in problems]
        probs = [(w.M, w.N, w.lam, w.band_k, g, P, T) for (w, g), P, T in zip(problems, Ps, Ths)]
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, reps = tomo.fit_batched(probs, precision=args.precision, concurrency=conc, autotune=autotune,
                                    eps_kkt=args.eps_kkt, max_newton=args.max_newton, **lim)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        return dt, st, reps

    # warm every code path (kernel configuration, graph capture) on one instance
    w0, g0 = problems[0]
    T0 = torch.empty(w0.M, w0.N, dtype=torch.float64, device="cuda")
    tomo.fit_batched([(w0.M, w0.N, w0.lam, w0.band_k, g0, Ps[0], T0)], precision=args.precision,
                     concurrency=1, eps_kkt=args.eps_kkt, max_newton=5)
    out = {"workload": f"c4 sample: {args.instances} instances x {len(W.C4_GAMMAS)} gammas, "
                       f"M ~ U{{256..{args.max_m}}}, N ~ U{{8..128}}, D = 2M",
           "solves": len(problems), "precision": args.precision, "data_s": t_data}
    fs = {}
    modes = [] if args.serial_sample > 0 else [(1, False)]
    modes.append((args.concurrency, False))
    if not args.no_autotune:
        modes.append((args.concurrency, True))
    for conc, tune in modes:
        dt, st, reps = run(conc, tune)
        key = f"conc{conc}_{'tuned' if tune else 'default'}"
        fs[key] = np.array([r["f"] for r in reps])
        out[key] = {"seconds": dt, "solves_per_s": len(problems) / dt,
                    "newton_iters": int(sum(r["iters_s1"] + r["iters_s2"] for r in reps)),
                    "cg_products": int(sum(r["cg_total"] for r in reps)),
                    "statuses": sorted(set(int(s) for s in st)),
                    "stops": {k: int(v) for k, v in zip(*np.unique([r["stop_name"] for r in reps],
                                                                    return_counts=True))},
                    "kkt_max": float(max(r["kkt"] for r in reps))}
        print(json.dumps({key: out[key]}), flush=True)
    ref = fs[f"conc{args.concurrency}_default"]
    if args.serial_sample > 0:
        # one-at-a-time solves of the first K problems against the pool's
        # results for the same problems
        k = min(args.serial_sample, len(problems))
        Ths = [torch.empty(problems[j][0].M, problems[j][0].N, dtype=torch.float64, device="cuda")
               for j in range(k)]
        probs = [(problems[j][0].M, problems[j][0].N, problems[j][0].lam, problems[j][0].band_k,
                  problems[j][1], Ps[j], Ths[j]) for j in range(k)]
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, reps = tomo.fit_batched(probs, precision=args.precision, concurrency=1,
                                    eps_kkt=args.eps_kkt, max_newton=args.max_newton, **lim)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        fk = np.array([r["f"] for r in reps])
        out["serial_sample"] = {"problems": k, "seconds": dt, "solves_per_s": k / dt,
                                "max_rel_objective_diff_vs_pool": float(np.max(np.abs(fk - ref[:k]) / ref[:k]))}
    else:
        ref = fs["conc1_default"]
    out["max_rel_objective_diff"] = float(max(np.max(np.abs(v - ref) / ref) for v in fs.values()))
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
