"""Training and evaluation of the learned warm start on the detector
population of `workloads.config_c5_instance` (M = 1024 photon numbers,
D = 2048 probes with lambda linear in [0, 768], up to 64 outcomes, gamma 1e-3):

    python -m paper_2404_02844_gb300.warmstart_eval [--train 2000] [--steps 3000]
        [--test 16] [--precision fp32] [--save weights.bin]

Trains on the simulator's true POVMs of `--train` instances (the solver's
optimum estimates exactly these), then solves `--test` held-out instances
from Theta^(0) = 1/N and from the network's Theta0 (fit_warm, with its
fallback) and prints one JSON line: training loss, held-out loss, Newton
iterations and solve time per start, and the objective agreement.
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
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tc", "fp64", "mixed"])
    ap.add_argument("--eps-kkt", type=float, default=1e-9)
    ap.add_argument("--save", default=None)
    args = ap.parse_args()

    import torch

    import paper_2404_02844_gb300 as tomo
    import workloads as W
    from paper_2404_02844_gb300 import build

    build.build()
    lam = W.probe_intensities(W.C5_D, W.C5_X)
    F = W.dense_poisson(W.C5_M, lam)
    t0 = time.perf_counter()
    Ptr, Ttr, nctr, _ = W.c5_batch(range(args.train), F=F)
    Pte, Tte, ncte, wte = W.c5_batch(range(100000, 100000 + args.test), F=F)
    t_data = time.perf_counter() - t0
    Ptr_d = torch.from_numpy(Ptr).cuda()
    Ttr_d = torch.from_numpy(Ttr).cuda()
    ws = tomo.WarmStart(W.C5_D, W.C5_C0, W.C5_M, max_batch=args.batch, seed=1)
    rng = np.random.default_rng(0)
    Pte_d = torch.from_numpy(Pte[:args.batch]).cuda()
    Tte_d = torch.from_numpy(Tte[:args.batch]).cuda()
    l_test0, _ = ws.loss_grad(Pte_d, Tte_d, ncte[:args.batch])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for s in range(args.steps):
        idx = torch.from_numpy(rng.choice(args.train, args.batch, replace=False)).cuda()
        losses.append(ws.train_step(Ptr_d[idx].contiguous(), Ttr_d[idx].contiguous(),
                                    nctr[idx.cpu().numpy()], lr=args.lr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    l_test1, _ = ws.loss_grad(Pte_d, Tte_d, ncte[:args.batch])
    if args.save:
        ws.save(args.save)

    rows = []
    for w in wte:
        with tomo.Plan.from_workload(w, precision=args.precision) as pl:
            P = torch.from_numpy(w.P).cuda()
            pl.fit(P, max_newton=2)  # warm the plan (graph capture) before timing
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Thc, rc = pl.fit(P, eps_kkt=args.eps_kkt, max_newton=3000)
            torch.cuda.synchronize()
            tc = time.perf_counter() - t0
            t0 = time.perf_counter()
            Thw, rw, used = tomo.fit_warm(pl, ws, P, eps_kkt=args.eps_kkt, max_newton=3000)
            torch.cuda.synchronize()
            tw = time.perf_counter() - t0
            fc, fw = pl.objective(P, Thc), pl.objective(P, Thw)
            uni = torch.full((w.M, w.N), 1.0 / w.N, dtype=torch.float64, device="cuda")
            f0w, f0u = pl.objective(P, ws.infer(P)), pl.objective(P, uni)
        rows.append(dict(N=w.N, cold_iters=rc["iters_s1"] + rc["iters_s2"],
                         warm_iters=rw["iters_s1"] + rw["iters_s2"], cold_s=tc, warm_s=tw,
                         used_warm=bool(used), rel_diff=(fw - fc) / fc, f0_warm_over_uniform=f0w / f0u))
    ci = np.array([r["cold_iters"] for r in rows])
    wi = np.array([r["warm_iters"] for r in rows])
    out = {
        "workload": "warm-start population: M=1024 D=2048 lambda lin [0,768], bins U{16..63}, "
                    "eta U[0.3,0.95], crosstalk U[0,1e-2], dark U[0,1e-3], 1e6 shots, gamma 1e-3",
        "params": ws.param_count, "train_instances": args.train, "steps": args.steps,
        "batch": args.batch, "lr": args.lr, "data_s": t_data, "train_s": t_train,
        "loss_first": losses[0], "loss_last_100": float(np.mean(losses[-100:])),
        "heldout_loss_before": l_test0, "heldout_loss_after": l_test1,
        "precision": args.precision, "test_instances": args.test,
        "cold_iters_mean": float(ci.mean()), "warm_iters_mean": float(wi.mean()),
        "cold_s_mean": float(np.mean([r["cold_s"] for r in rows])),
        "warm_s_mean": float(np.mean([r["warm_s"] for r in rows])),
        "used_warm": int(sum(r["used_warm"] for r in rows)),
        "max_rel_objective_diff": float(max(abs(r["rel_diff"]) for r in rows)),
        "f0_warm_over_uniform_median": float(np.median([r["f0_warm_over_uniform"] for r in rows])),
        "rows": rows,
    }
    print(json.dumps(out), flush=True)
    ws.close()


if __name__ == "__main__":
    main()
